"""GB300-native k-d tree queries (fcp / kNN over left-balanced, level-order
trees, stack-free traversal after Wald, arXiv 2210.12859)."""
