// Instantiation of the node-model kernels for the Dint model.
#include "model_dint.cuh"
#include "node_kernels.cuh"

namespace ocpg {
ocp_status node_eval_dint(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  return node_eval_dispatch<Dint, TILE_DINT>(h, out, c, s);
}
ocp_status node_prod_dint(ocp* h, const ProdCall& c, cudaStream_t s) { return node_prod_dispatch<Dint, TILE_DINT>(h, c, s); }
}  // namespace ocpg
