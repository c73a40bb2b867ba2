// All device models of the dynamics x' = f(x, u) (paper Sec. 3), for the translation units
// that need every model's tables (pattern compiler, batch, objective kernels).
#pragma once
#include "model_base.cuh"
#include "model_vdp.cuh"
#include "model_dint.cuh"
#include "model_cartpole.cuh"
#include "model_goddard.cuh"
#include "model_quad.cuh"
