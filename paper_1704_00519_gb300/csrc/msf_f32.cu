// msf_f32.cu -- FP32-bulk instantiation: WENO5 fluxes, primitive recovery,
// ghost states, HLLC and the CFL bound in float; conserved state, flux
// accumulation and the RK update stay FP64.
#include "msf_kernels.cuh"
#include "msf_ops.h"
#include "msf_prec.inc"
#include "msf_adjoint.cuh"
#include "msf_tiled.cuh"

namespace msf {
const Ops* ops_f32() {
  static const Ops ops = make_ops<float>();
  return &ops;
}
const AdjOps* adj_ops_f32() {
  static const AdjOps ops = make_adj_ops<float>();
  return &ops;
}
const TiledOps* tiled_ops_f32() {
  static const TiledOps ops = make_tiled_ops<float>();
  return &ops;
}
}  // namespace msf
