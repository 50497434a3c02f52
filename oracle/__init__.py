"""FP64 CPU oracle (test infrastructure only; see ``fdl_oracle``)."""
