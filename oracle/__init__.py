"""CPU oracle of the method (test infrastructure only; see msf_oracle.c)."""
