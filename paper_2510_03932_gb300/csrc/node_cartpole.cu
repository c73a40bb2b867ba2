// Instantiation of the node-model kernels for the CartPole model.
#include "model_cartpole.cuh"
#include "node_kernels.cuh"

namespace ocpg {
ocp_status node_eval_cartpole(ocp* h, unsigned out, const EvalCall& c, cudaStream_t s) {
  return node_eval_dispatch<CartPole, TILE_CARTPOLE>(h, out, c, s);
}
ocp_status node_prod_cartpole(ocp* h, const ProdCall& c, cudaStream_t s) { return node_prod_dispatch<CartPole, TILE_CARTPOLE>(h, c, s); }
}  // namespace ocpg
