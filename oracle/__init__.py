"""FP64 CPU oracle (test infrastructure only; see sph_oracle.h)."""
