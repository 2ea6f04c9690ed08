"""GB300-native covariance-free EM (CoFEM) for sparse Bayesian learning."""
