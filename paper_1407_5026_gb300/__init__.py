"""GB300-native parallel-rejection kinetic Monte Carlo for the lattice Coulomb glass."""
