// Instantiation of the node-model kernels for the quadrotor model.
#include "model_quad.cuh"
#include "node_kernels.cuh"

namespace ocpg {
ocp_status node_eval_quad(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  return node_eval_dispatch<Quadrotor, TILE_QUAD_EVAL>(h, out, c, s);
}
ocp_status node_prod_quad(ocp* h, const ProdCall& c, cudaStream_t s) {
  return node_prod_dispatch<Quadrotor, TILE_QUAD>(h, c, s);
}
}  // namespace ocpg
