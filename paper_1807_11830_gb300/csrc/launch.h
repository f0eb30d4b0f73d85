// Host-side launchers of the SENSE kernels, dispatched on the transform
// length.  Each returns cudaErrorInvalidValue for a length without a
// compiled configuration, else the launch status.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "persistent.cuh"

namespace sense {

bool size_supported(int n);
int col_width(int n);      // columns per block of the column kernels for length n
int col_threads(int n);
int row_width(int n);      // rows per block of the row kernels for length n

template <class St>
cudaError_t launch_fwd_col(int n, const FwdColArgs<St>& a, int tiles, int frames, cudaStream_t s);
template <class St>
cudaError_t launch_adj_col(int n, int mode, const AdjColArgs<St>& a, int tiles, int frames, cudaStream_t s);
// normal operator, kernel variant `variant` (0 .. kNormVariants-1; see NormCfg);
// the grid's tile count follows the variant's tile width
template <class St>
cudaError_t launch_normal(int n, int variant, bool cg, const NormalArgs<St>& a, int frames, cudaStream_t s);
// tile width / threads per block of a normal-operator variant, 0 if it does not exist
int normal_variant_width(int n, int variant);
int normal_variant_threads(int n, int variant);
// 1 if the variant reads the transposed maps S^T [C][nx][ny] (lane-major tiles)
int normal_variant_transposed(int n, int variant);
// S [C][ny][nx] -> S^T [C][nx][ny] in storage type (bf16 pairs or complex64)
cudaError_t launch_transpose_maps(bool bf16, const void* S, void* ST, int ny, int nx, int coils, cudaStream_t s);
// persistent CG kernel (all iterations of all frames of `a` in one launch,
// `sms` x resident blocks per SM)
template <class St>
cudaError_t launch_cg_persistent(int n, int variant, const PArgs& a, int sms, cudaStream_t s);
// blocks per SM the persistent CG kernel of (n, variant, storage) keeps
// resident (0 if the variant does not exist)
int cg_persistent_resident(int n, int variant, bool bf16);
// forward row pass: FP32 in, storage St out
template <class St>
cudaError_t launch_rows_fwd(int n, const RowArgs<float2, typename St::T>& a, cudaStream_t s);
// inverse row pass: storage St in, FP32 out
template <class St>
cudaError_t launch_rows_inv(int n, const RowArgs<typename St::T, float2>& a, cudaStream_t s);

// TMA-staged persistent column passes (one wave of resident blocks looping
// over (frame, column tile) items).  cudaErrorNotSupported when the length
// has none or its tiles do not fit shared memory: the caller then uses the
// register-staged kernels above.  tmK: the intermediate [F*C*L][nx] float2,
// box 8 x kbox_rows(L); tmS: S [C*ny][nx] in storage type, box 8 x
// min(ny, ny/2 when ny > 256).
bool coltma_supported(int n);
template <class St>
cudaError_t launch_adj_col_tma(int n, int mode, const CUtensorMap& tmK, const CUtensorMap& tmS,
                               const AdjColArgs<St>& a, int frames, int sms, cudaStream_t s);
template <class St>
cudaError_t launch_fwd_col_tma(int n, const CUtensorMap& tmS, const FwdColArgs<St>& a, int tiles, int frames,
                               int sms, cudaStream_t s);

// Single-launch fused operators (square images with a TMA column pass; else
// cudaErrorNotSupported): E^H / CG start / RSS (`mode` 0 / 1 / 2; for RSS, St
// is complex64 and y_bf16 gives y's storage) and E.  `sc` holds the ticket and
// per-frame counters, zeroed by the caller on the same stream.
struct FusedSched;
template <class St>
cudaError_t launch_adjoint_fused(int n, int mode, bool y_bf16, const CUtensorMap& tmK, const CUtensorMap& tmS,
                                 const AdjColArgs<St>& a, const void* y, float2* tmp_out, const FusedSched& sc,
                                 float cs, int sms, cudaStream_t s);
template <class St>
cudaError_t launch_forward_fused(int n, const CUtensorMap& tmS, const FwdColArgs<St>& a, void* y, const FusedSched& sc,
                                 float cs, int sms, cudaStream_t s);

// Set the dynamic shared memory limit of `kern` once per device.
template <class K>
inline cudaError_t ensure_smem(K kern, size_t bytes, unsigned long long* done_mask) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(done_mask, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) __atomic_fetch_or(done_mask, bit, __ATOMIC_ACQ_REL);
  return e;
}

}  // namespace sense
