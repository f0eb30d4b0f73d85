// CG vector update, CG finish and bf16 conversion kernels (host-launched by
// the API unit only).
#pragma once
#include "common.cuh"

namespace sense {

// ---------------------------------------------------------------------------
// CG vector update: x += alpha p, r -= alpha q, <r, r>, then beta and the
// stopping test in the last block of each frame.
// ---------------------------------------------------------------------------
constexpr int UPD_THREADS = 256;
constexpr int UPD_VEC = 4;  // float4 (two complex values) per thread and step
constexpr int UPD_PER_BLOCK = UPD_THREADS * UPD_VEC * 2;  // complex values per block

struct UpdateArgs {
  float4* x;
  const float4* p;
  const float4* q;
  float4* r;
  long img4;   // float4 per image
  int blocks_per_frame;
  CgState cg;
};

__global__ void __launch_bounds__(UPD_THREADS) k_cg_update(UpdateArgs a) {
  const int f = blockIdx.y;
  if (a.cg.active[f] == 0) return;
  __shared__ double red[32];
  const float al = (float)__ldg(a.cg.alpha + f);
  const size_t base = (size_t)f * a.img4;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < UPD_VEC; ++j) {
    const long i = (long)blockIdx.x * (UPD_THREADS * UPD_VEC) + j * UPD_THREADS + threadIdx.x;
    if (i < a.img4) {
      float4 xv = a.x[base + i];
      const float4 pv = __ldg(a.p + base + i);
      const float4 qv = __ldg(a.q + base + i);
      float4 rv = a.r[base + i];
      xv.x = fmaf(al, pv.x, xv.x); xv.y = fmaf(al, pv.y, xv.y);
      xv.z = fmaf(al, pv.z, xv.z); xv.w = fmaf(al, pv.w, xv.w);
      rv.x = fmaf(-al, qv.x, rv.x); rv.y = fmaf(-al, qv.y, rv.y);
      rv.z = fmaf(-al, qv.z, rv.z); rv.w = fmaf(-al, qv.w, rv.w);
      a.x[base + i] = xv;
      a.r[base + i] = rv;
      acc = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, acc))));
    }
  }
  const double tot = block_sum<UPD_THREADS>((double)acc, red);
  const CgState& g = a.cg;
  double* slot = g.part + (size_t)f * g.part_stride + blockIdx.x;
  if (publish_and_arrive(tot, slot, g.counter + f, (unsigned)a.blocks_per_frame)) {
    const double rho_new = ordered_sum(g.part + (size_t)f * g.part_stride, a.blocks_per_frame);
    g.counter[f] = 0u;
    const double rho0 = g.rho0[f];
    g.iters[f] += 1;
    g.resid[f] = sqrt(rho_new / rho0);
    const bool stop = (rho_new == 0.0) || (g.tol > 0.0 && sqrt(rho_new / rho0) <= g.tol);
    if (stop) {
      g.active[f] = 0;
      g.outcome[f] = CG_CONVERGED;
      atomicSub(g.live, 1);
    } else {
      g.beta[f] = rho_new / g.rho[f];
    }
    g.rho[f] = rho_new;
  }
}

// Final per-frame outputs of a CG solve.
__global__ void k_cg_finish(CgState g, int frames, int* iters_out, double* resid_out, int* outcome_out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= frames) return;
  int oc = g.outcome[f];
  if (oc == CG_RUNNING) oc = CG_MAXITER;
  g.outcome[f] = oc;
  if (iters_out) iters_out[f] = g.iters[f];
  if (resid_out) resid_out[f] = g.resid[f];
  if (outcome_out) outcome_out[f] = oc;
}

__global__ void k_to_bf16(const float2* in, __nv_bfloat162* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float22bfloat162_rn(in[i]);
}

}  // namespace sense
