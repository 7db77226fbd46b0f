"""GB300-native Exchange Monte Carlo for the 3D Random Field Ising Model (placeholder)."""
