"""GB300-native tensor-product multigrid preconditioned CG (arXiv:1408.2981)."""
