// wo_zops_a.cu - fused z pass instantiations with equal or growing volume
// counts (reconstruct and adjoint: channels -> properties), and the 2D solve.
#include "wo_zops.cuh"

namespace wo {

#define WO_Z_SWITCH(NI, NO)                                                   \
  switch (Z) {                                                                \
    WO_FOR_EACH_SIZE(WO_Z_CASE_##NI##NO)                                      \
    default:                                                                  \
      return cudaErrorInvalidValue;                                           \
  }
#define WO_Z_CASE_11(n) case n: return launch_z_fused<n, 1, 1>(in, out, tf, op, nt, Y, Xh, s);
#define WO_Z_CASE_12(n) case n: return launch_z_fused<n, 1, 2>(in, out, tf, op, nt, Y, Xh, s);
#define WO_Z_CASE_22(n) case n: return launch_z_fused<n, 2, 2>(in, out, tf, op, nt, Y, Xh, s);
#define WO_Z_CASE_23(n) case n: return launch_z_fused<n, 2, 3>(in, out, tf, op, nt, Y, Xh, s);

cudaError_t z_fused_grow(int ni, int no, int Z, const float2* in, float2* out, const float2* tf, ZOp op, int nt,
                         int Y, int Xh, cudaStream_t s) {
  if (ni == 1 && no == 1) { WO_Z_SWITCH(1, 1) }
  if (ni == 1 && no == 2) { WO_Z_SWITCH(1, 2) }
  if (ni == 2 && no == 2) { WO_Z_SWITCH(2, 2) }
  if (ni == 2 && no == 3) { WO_Z_SWITCH(2, 3) }
  return cudaErrorNotSupported;
}

#define WO_S_CASE_1(n) case n: return launch_z_solve2d<n, 1>(in, out, tf, op, nt, Y, Xh, s);
#define WO_S_CASE_2(n) case n: return launch_z_solve2d<n, 2>(in, out, tf, op, nt, Y, Xh, s);

cudaError_t z_solve2d(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int nt, int Y, int Xh,
                      cudaStream_t s) {
  if (op.n_in == 1) {
    switch (Z) {
      WO_FOR_EACH_SIZE(WO_S_CASE_1)
      default: return cudaErrorInvalidValue;
    }
  }
  if (op.n_in == 2) {
    switch (Z) {
      WO_FOR_EACH_SIZE(WO_S_CASE_2)
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorNotSupported;
}

}  // namespace wo
