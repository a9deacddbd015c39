"""FP64 CPU parity oracle (test infrastructure only; see oracle/oracle.c)."""
