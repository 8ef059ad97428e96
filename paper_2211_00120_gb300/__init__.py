"""GB300-native left-balanced k-d tree construction (Wald, arXiv 2211.00120)."""
