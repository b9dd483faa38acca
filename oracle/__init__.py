"""CPU oracle of the Metropolis film sweeps — test infrastructure only (see isf_oracle.h)."""
