// Instantiation of the node-model kernels for the VdP model.
#include "model_vdp.cuh"
#include "node_kernels.cuh"

namespace ocpg {
ocp_status node_eval_vdp(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  return node_eval_dispatch<VdP, TILE_VDP>(h, out, c, s);
}
ocp_status node_prod_vdp(ocp* h, const ProdCall& c, cudaStream_t s) { return node_prod_dispatch<VdP, TILE_VDP>(h, c, s); }
}  // namespace ocpg
