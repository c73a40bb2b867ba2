// Launch shapes and compile-time tables shared by the kernels and the host code that lays out
// their outputs (the kernels' FP64 instruction counts depend on this file, not on the handle).
#pragma once

namespace ocpg {

// Threads (= nodes) per CTA of the node-model kernels; a tile owns TILE-1 nodes.
constexpr int TILE_VDP = 256, TILE_CARTPOLE = 128, TILE_DINT = 256, TILE_QUAD = 64;
// The quadrotor's evaluation kernels (F, c, g, J, H and the fused step) run 128-node tiles with
// three CTAs per SM at its register cap, its product kernels 64-node tiles (measured at N = 1e6:
// fused step 846 -> 832 us, evaluation 533 -> 512 us; the products gain nothing from the larger
// tile and lose up to 5% at N = 1e5).  Every output is per node but the objective, whose tile
// sums only the evaluation kernels form.
constexpr int TILE_QUAD_EVAL = 128;
// Most state components with a time-varying reference (node models have at most 9 states).
constexpr int kMaxTrack = 16;
// Nodes per CTA of the heat-equation kernels (one per lane); a tile owns 31 nodes.
constexpr int HEAT_TILE_NODES = 32;

// Output selection bits of the fused evaluation kernels.
enum : unsigned { O_F = 1u, O_C = 2u, O_G = 4u, O_J = 8u, O_H = 16u, O_ALL = 31u,
                  // products evaluated in the same pass (the fused step)
                  O_JV = 32u, O_JTV = 64u, O_HV = 128u, O_STEP = 255u };

// Per-component Jacobian row template (local variable indices), as read from the model.
constexpr int RT_XV = 6, RT_UV = 4;
constexpr int RT_STRIDE = 2 + RT_XV + RT_UV;  // ints per row in the device table: rx, ru, xv[], uv[]
struct RowTemplate {
  int rx = 0, ru = 0;
  int xv[RT_XV] = {-1, -1, -1, -1, -1, -1};
  int uv[RT_UV] = {-1, -1, -1, -1};
  bool jz[RT_XV] = {};  // entry xv[e] is the identity term alone (df_k/dx_v identically zero)
  int count() const { return 2 * (rx + ru); }
};

}  // namespace ocpg
