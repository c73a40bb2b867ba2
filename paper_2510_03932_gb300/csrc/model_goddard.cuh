// Device model of the Goddard rocket (sparsity tables) dynamics (the conventions of every model are stated in
// model_base.cuh).
#pragma once
#include "model_base.cuh"

namespace ocpg {

// ------------------------------------------------------------------------------------
// Goddard rocket (the paper's first benchmark problem, appendix): z = (r, v, m, u) =
// (altitude, speed, mass, normalised thrust), params (Cd, beta, Tmax, b):
//   r' = v,  v' = -D - 1/r^2 + u Tmax / m,  m' = -b Tmax u,  D = Cd v^2 exp(-beta (r - 1)) / m.
// Only the sparsity tables live here (for the pattern compiler); the values are computed by
// the dedicated free-final-time kernels (goddard_kernels.cu).
// ------------------------------------------------------------------------------------
struct Goddard {
  static constexpr int EVAL_MIN_CTAS = 0;
  static constexpr int NX = 3, NU = 1, NZ = 4;
  static constexpr int MAXRX = 3, MAXRU = 1;
  OCP_TABLE1(RX, int, NX, {2, 3, 1})
  OCP_TABLE1(RU, int, NX, {0, 1, 1})
  OCP_TABLE2(XV, int, NX, MAXRX, {{0, 1, -1}, {0, 1, 2}, {2, -1, -1}})
  OCP_TABLE2(UV, int, NX, MAXRU, {{-1}, {0}, {0}})
  OCP_TABLE2(JZ, bool, NX, MAXRX, {{true, false, false}, {false, false, false}, {true, false, false}})
  OCP_TABLE1(HK, bool, NX, {false, true, false})
  static constexpr int NHD = 7;
  OCP_TABLE1(HA, int, NHD, {0, 1, 1, 2, 2, 2, 3})
  OCP_TABLE1(HB, int, NHD, {0, 0, 1, 0, 1, 2, 2})
};

}  // namespace ocpg
