"""GB300-native 3-center Coulomb integrals and density-fitted J (arXiv:2210.03192 hot path)."""
