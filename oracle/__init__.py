"""CPU oracle (test infrastructure only; see ocp_oracle.cpp)."""
