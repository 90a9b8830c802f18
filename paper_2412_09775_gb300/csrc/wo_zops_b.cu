// wo_zops_b.cu - fused z pass instantiations with shrinking volume counts
// (forward model: properties -> channels), and the dispatcher.
#include "wo_zops.cuh"

namespace wo {

cudaError_t z_fused_grow(int ni, int no, int Z, const float2* in, float2* out, const float2* tf, ZOp op, int nt,
                         int Y, int Xh, cudaStream_t s);

#define WO_Z_CASE_21(n) case n: return launch_z_fused<n, 2, 1>(in, out, tf, op, nt, Y, Xh, s);
#define WO_Z_CASE_32(n) case n: return launch_z_fused<n, 3, 2>(in, out, tf, op, nt, Y, Xh, s);

cudaError_t z_fused(int Z, const float2* in, float2* out, const float2* tf, ZOp op, int nt, int Y, int Xh,
                    cudaStream_t s) {
  if (z_reg_supported(Z, op)) return z_fused_reg(Z, in, out, tf, op, nt, Y, Xh, s);
  if (op.n_in == 2 && op.n_out == 1) {
    switch (Z) {
      WO_FOR_EACH_SIZE(WO_Z_CASE_21)
      default: return cudaErrorInvalidValue;
    }
  }
  if (op.n_in == 3 && op.n_out == 2) {
    switch (Z) {
      WO_FOR_EACH_SIZE(WO_Z_CASE_32)
      default: return cudaErrorInvalidValue;
    }
  }
  return z_fused_grow(op.n_in, op.n_out, Z, in, out, tf, op, nt, Y, Xh, s);
}

}  // namespace wo
