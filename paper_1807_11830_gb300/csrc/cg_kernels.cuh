// CG vector update, CG finish and bf16 conversion kernels (host-launched by
// the API unit only).
#pragma once
#include "persistent.cuh"

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
  float4* __restrict__ xp = a.x + base;
  float4* __restrict__ rp = a.r + base;
  const float4* __restrict__ pp = a.p + base;
  const float4* __restrict__ qp = a.q + base;
  // issue every load before any store so they are all in flight together
  float4 xv[UPD_VEC], pv[UPD_VEC], qv[UPD_VEC], rv[UPD_VEC];
  const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < UPD_VEC; ++j) {
    const long i = (long)blockIdx.x * (UPD_THREADS * UPD_VEC) + j * UPD_THREADS + threadIdx.x;
    const bool ok = i < a.img4;
    xv[j] = ok ? xp[i] : z;
    pv[j] = ok ? __ldg(pp + i) : z;
    qv[j] = ok ? __ldg(qp + i) : z;
    rv[j] = ok ? rp[i] : z;
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < UPD_VEC; ++j) {
    const long i = (long)blockIdx.x * (UPD_THREADS * UPD_VEC) + j * UPD_THREADS + threadIdx.x;
    float4 xn = xv[j], rn = rv[j];
    xn.x = fmaf(al, pv[j].x, xn.x); xn.y = fmaf(al, pv[j].y, xn.y);
    xn.z = fmaf(al, pv[j].z, xn.z); xn.w = fmaf(al, pv[j].w, xn.w);
    rn.x = fmaf(-al, qv[j].x, rn.x); rn.y = fmaf(-al, qv[j].y, rn.y);
    rn.z = fmaf(-al, qv[j].z, rn.z); rn.w = fmaf(-al, qv[j].w, rn.w);
    if (i < a.img4) {
      xp[i] = xn;
      rp[i] = rn;
      acc = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, fmaf(rn.z, rn.z, fmaf(rn.w, rn.w, acc))));
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
// Per-frame CG outputs; `coupled`: all frames report the group's (slot 0).
__global__ void k_cg_finish(CgState g, int frames, int* iters_out, double* resid_out, int* outcome_out,
                            int coupled) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= frames) return;
  const int s = coupled ? 0 : f;
  int oc = g.outcome[s];
  if (oc == CG_RUNNING) oc = CG_MAXITER;
  if (!coupled) g.outcome[f] = oc;
  if (iters_out) iters_out[f] = g.iters[s];
  if (resid_out) resid_out[f] = g.resid[s];
  if (outcome_out) outcome_out[f] = oc;
}

// Frames coupled into one CG: after the per-frame CG start, slot 0 takes the
// group's start state, rho0 = sum over frames (in frame order).
__global__ void k_cg_couple_start(CgState g, int frames) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rho = 0.0;
  for (int f = 0; f < frames; ++f) rho += g.rho[f];
  g.rho[0] = rho;
  g.rho0[0] = rho;
  g.iters[0] = 0;
  g.alpha[0] = 0.0;
  g.beta[0] = 0.0;
  const bool run = rho > 0.0 && isfinite(rho);  // not finite: NaN/Inf input, breakdown with residual NaN
  g.active[0] = run ? 1 : 0;
  g.outcome[0] = run ? CG_RUNNING : (rho == 0.0 ? CG_CONVERGED : CG_BREAKDOWN);
  g.resid[0] = run ? 1.0 : (rho == 0.0 ? 0.0 : rho - rho);
}

// CG iterates of a centred-k-space problem live in the modulated space
// x' = D x (D = diag((-1)^(y+x))): map the solution back, in place.
__global__ void k_checkerboard(float2* x, int ny, int nx, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long pix = i % ((long)ny * nx);
  const int yy = (int)(pix / nx), xx = (int)(pix - (long)yy * nx);
  if ((yy + xx) & 1) {
    const float2 v = x[i];
    x[i] = make_float2(-v.x, -v.y);
  }
}

// Self-test of the bounded wait: waits for a flag that nothing sets and
// records whether the wait gave up (1) or saw the flag (0).
__global__ void k_wait_selftest(const int* flag, long max_spins, int* timed_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *timed_out = wait_at_least(flag, 1, max_spins) ? 0 : 1;
}

__global__ void k_to_bf16(const float2* in, __nv_bfloat162* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = __float22bfloat162_rn(in[i]);
}

}  // namespace sense
