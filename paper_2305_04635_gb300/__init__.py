"""GB300-native banded Cholesky factorization and solve (arXiv 2305.04635)."""
