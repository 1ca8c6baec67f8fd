"""FP64 CPU oracle of the HOTRG step (test infrastructure only; see hotrg_oracle)."""
