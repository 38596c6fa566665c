"""GB300-native ORAS-GMRES solver for the 27-point finite-difference Helmholtz problem."""
