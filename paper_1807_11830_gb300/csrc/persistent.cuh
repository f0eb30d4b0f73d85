// Persistent CG-SENSE iteration kernel: one launch runs every CG iteration of
// every frame in a table.
//
// Work is cut into items, handed out in a fixed order by one global atomic
// ticket counter:
//   ticket -> (iteration k, phase, frame f, piece)
//   phase 0 (normal): piece = column tile: p_k = r + beta p_{k-1},
//                     q = E^H E p_k on the tile, Re<p_k, q> partial;
//                     the last tile of frame f computes alpha (or freezes f).
//   phase 1 (update): piece = chunk of the image: x += alpha p_k,
//                     r -= alpha q, <r, r> partial; the last chunk computes
//                     beta and the stopping test.
// Tickets follow one of two orders (PArgs::lag, below): iteration-major
// (iteration, then phase, then frame, then piece), or frame-staggered, where
// a frame's update chunks come a few frames' worth of tiles after its own
// tiles, so they rarely find those tiles still running.  In both, an item
// waits (thread 0, bounded spin) only for the previous phase of its own
// frame, i.e. for items with smaller tickets, which blocks already running
// have taken.  So the wait always ends; frames pipeline freely: one frame's
// memory-bound update runs while another frame's transform-bound normal
// product fills the rest of the GPU, and no kernel boundary or launch tail
// separates the phases.  A wait that exceeds its bound sets ERR_TIMEOUT,
// skips the item's work and still counts the item, so the launch ends.
//
// Data written by other blocks of the launch (p, r, q, x, partials, scalars)
// is read through L2 (ld.global.cg / acquire) and written through L2.
#pragma once
#include "kernels.cuh"

namespace sense {

// A two-phase item of a frame-staggered order: units 0 .. U-1 (frames, or
// frame-iterations) each have P1 first-phase items and P2 second-phase ones.
struct StaggeredItem {
  int second;  // 0: first phase, 1: second phase
  int unit;
  int piece;
};

// Ticket t of the frame-staggered order with lag D: stage s holds the
// first-phase items of unit s (s < U), then the second-phase items of unit
// s - D (s >= D).  So the first min(D, U) stages hold first-phase items only,
// stages D .. U - 1 both kinds, and the last min(D, U) stages second-phase
// items only.  A unit's second phase comes D stages after its first.
__host__ __device__ __forceinline__ StaggeredItem staggered_item(long t, int U, int P1, int P2, int D) {
  StaggeredItem it;
  const long A = D < U ? D : U;
  if (t < A * P1) {
    it.second = 0;
    it.unit = (int)(t / P1);
    it.piece = (int)(t - (long)it.unit * P1);
    return it;
  }
  t -= A * P1;
  const long M = U > D ? U - D : 0;
  const long per = (long)P1 + P2;
  if (t < M * per) {
    const long s = D + t / per;
    const int r = (int)(t - (s - D) * per);
    it.second = r >= P1;
    it.unit = it.second ? (int)(s - D) : (int)s;
    it.piece = it.second ? r - P1 : r;
    return it;
  }
  t -= M * per;
  it.second = 1;
  it.unit = (int)((U - A) + t / P2);
  it.piece = (int)(t - (long)(it.unit - (U - A)) * P2);
  return it;
}

// Update items: each thread updates kUpdateRounds rounds of kUpdateVec float4
// (two complex values each) of one frame's image.
constexpr int kUpdateVec = 4, kUpdateRounds = 16;
__host__ __device__ constexpr int update_chunks(size_t img, int threads) {
  return (int)((img / 2 + (size_t)threads * kUpdateVec * kUpdateRounds - 1) /
               ((size_t)threads * kUpdateVec * kUpdateRounds));
}

// Item orders of the persistent CG kernel (PArgs::lag).
//   kOrderIterationMajor: per CG iteration, every frame's normal-product
//     tiles, then every frame's update chunks.
//   D >= 0: frame-staggered over frame-iterations u = k F + f
//     (staggered_item with P1 = tiles, P2 = chunks): u's update chunks follow
//     the tiles of u + D.  Valid when every frame is its own CG (no temporal
//     coupling) and D < F: u's update waits for u's tiles, D stages earlier,
//     and the tiles of u + F (the frame's next iteration) wait for u's
//     update, F - D stages earlier.  So every wait is for smaller tickets.
//   kOrderAuto: the launcher picks D from the grid: enough stages that about
//     one wave of tiles separates a frame's tiles from its update.
constexpr int kOrderIterationMajor = -1, kOrderAuto = -2;
__host__ __device__ constexpr int persistent_lag(int frames, int tiles, int grid) {
  const int d = (grid + tiles - 1) / (tiles > 0 ? tiles : 1) + 1;
  return frames <= 1 ? 0 : (d < frames - 1 ? d : frames - 1);
}

// One frame of the table: its instance's maps, its own vectors and its own
// CG scalars (wherever its owner keeps them), so frames of different
// problems can share one launch.
struct PFrame {
  const void* S;       // maps [C][N][nx] of the frame's instance (storage type)
  const int* lines;    // this frame's lines [L]
  float2* x;           // [N][nx] image (output)
  float2* r;           // residual
  float2* p[2];        // search directions, ping-pong by global iteration parity
  float2* q;           // E^H E p
  double *rho, *rho0, *alpha, *beta, *resid;
  int *iters, *outcome, *active;
  int coils, L;
  const void* tmap;    // TMA descriptor of S ([C*N] rows x nx, box W x min(N, N/2 if N > 256))
  int k0;              // CG iterations this frame has already done before the launch
  int kmax;            // the frame does no work at global iterations >= kmax
  double tol;          // relative-residual stopping tolerance (0: none)
  float lambda;        // Tikhonov weight: the frame solves (E^H E + lambda I) x = E^H y
  // Frames coupled in time share one CG: the group is the table range
  // [g0, g0 + gsize) (g0 = own index, gsize = 1 for an independent frame),
  // whose scalars live at the first frame's slots; arrivals, ready flags and
  // partial sums are counted over the whole group.  lambda_t weighs the
  // cyclic temporal second difference with the table entries nb_prev, nb_next.
  int g0, gsize;
  float lambda_t;
  int nb_prev, nb_next;
};

// (Members of a frame entry are picked with constant indices throughout: a
// runtime index into the kernel's copy of the entry would put the copy in
// local memory.)
struct PState {
  unsigned *nrm_arrive, *upd_arrive;          // [frames] arrivals of the current phase
  int *nrm_ready, *upd_ready;                 // [frames] launch iterations whose phase is complete
  double *part_nrm, *part_upd;                // [frames][tiles] / [frames][chunks]
};

// The order a frame table allows: the staggered one (picked by the launcher)
// unless some frames are coupled in time.
inline int persistent_order(const PFrame* host_table, int frames) {
  for (int f = 0; f < frames; ++f)
    if (host_table[f].gsize != 1) return kOrderIterationMajor;
  return kOrderAuto;
}

struct PArgs {
  const PFrame* frames;
  int nframes, nx, tiles, chunks, iters;
  int lag;  // item order: kOrderIterationMajor, kOrderAuto or a stagger D >= 0 (see above)
  unsigned* ticket;
  const float2* tw;  // twiddles of the column transform
  int* err;
  PState st;
};

constexpr long kPersistentMaxSpins = 1L << 24;  // x >= 64 ns sleeps: a wait gives up after >= 1 s

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0: wait until *flag >= target.  Returns false after max_spins polls.
__device__ __forceinline__ bool wait_at_least(const int* flag, int target, long max_spins = kPersistentMaxSpins) {
  long spins = 0;
  while (ld_acquire(flag) < target) {
    if (++spins > max_spins) return false;
    __nanosleep(64);
  }
  return true;
}

// Shared memory of the persistent kernel.  Block-tile configurations: two
// TMA map tiles, the column kernels' layout, two mbarriers.  Lane-major
// configurations: the layout of normal_tile_warp.
template <class C, class St>
__host__ __device__ constexpr size_t persistent_smem_bytes() {
  if constexpr (is_wcol<C>::value)
    return wcol_smem_bytes<C, St>();
  else
    return 2 * (size_t)C::N * C::W * sizeof(typename St::T) + ((col_smem_bytes_c<C>() + 7) & ~(size_t)7) + 16;
}

// The normal-product piece of the persistent kernel for each engine: set-up
// at block start, the line map of a frame, and one tile.
template <class C, class St, bool WARP = is_wcol<C>::value>
struct PTile;

template <class C, class St>
struct PTile<C, St, false> {  // block tiles, maps staged by TMA as [N][W] tiles
  SStage<C, St> sg;
  ColSmem s;
  __device__ __forceinline__ PTile(unsigned char* smem, const float2* tw) {
    constexpr size_t SB = (size_t)C::N * C::W * sizeof(typename St::T);
    sg.buf[0] = reinterpret_cast<typename St::T*>(smem);
    sg.buf[1] = reinterpret_cast<typename St::T*>(smem + SB);
    s = col_smem_c<C>(smem + 2 * SB);
    sg.bar = reinterpret_cast<uint64_t*>(smem + 2 * SB + ((col_smem_bytes_c<C>() + 7) & ~(size_t)7));
    for (int i = threadIdx.x; i < C::N; i += C::THREADS) s.tw[i] = tw[i];
    if (threadIdx.x == 0) {
      mbar_init(sg.bar, 1);
      mbar_init(sg.bar + 1, 1);
      mbar_fence_init();
    }
  }
  __device__ __forceinline__ double* red() const { return s.red; }
  // called before the line map is built, so the first coil's copy overlaps it
  __device__ __forceinline__ void prefetch(const PFrame& fr, int piece, unsigned nfill) {
    sg.tmap = fr.tmap;
    if (threadIdx.x == 0) sg.issue(nfill, piece, 0);
  }
  // the tile builds the line map while its p loads are in flight
  __device__ __forceinline__ float run(const NormalTile& nt, const int* lines, int L, unsigned nfill, int* err) const {
    return normal_tile_tma<C, St>(nt, s, 0u, sg, nfill, err, lines, L);
  }
};

template <class C, class St>
struct PTile<C, St, true> {  // lane-major tiles, maps by per-warp bulk copies of S^T
  WSmem<C, St> s;
  __device__ __forceinline__ PTile(unsigned char* smem, const float2* tw) : s(wcol_smem<C, St>(smem)) {
    wcol_setup<C, St>(s, tw);
  }
  __device__ __forceinline__ double* red() const { return s.red; }
  __device__ __forceinline__ void prefetch(const PFrame&, int, unsigned) {}
  // the tile builds the line map while its p staging loads are in flight
  __device__ __forceinline__ float run(const NormalTile& nt, const int* lines, int L, unsigned nfill, int* err) const {
    return normal_tile_warp<C, St, true>(nt, s, 0u, nfill, err, lines, L);
  }
};

template <int N, int V, class St, int TH = NormCfg<N, V>::C::THREADS, int MINB = NormCfg<N, V>::MINB>
__global__ void __launch_bounds__(TH, MINB) k_cg_persistent(PArgs a) {
  using C = typename NormCfg<N, V>::C;
  constexpr int T = C::THREADS;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PTile<C, St> tile(smem_raw, a.tw);
  __shared__ int s_ticket, s_ok, s_active;
  unsigned nfill = 0;  // map copies requested so far by this block (same in every thread)
  // The thread that takes the block's tickets: the next item's ticket is
  // taken at the end of the current item, while the block's threads wait at
  // their fence for their stores to become visible, so its round trip
  // overlaps that wait.
  constexpr int TK = T > 32 ? 32 : 0;
  if (threadIdx.x == TK) s_ticket = (int)atomicAdd(a.ticket, 1u);

  const int per_iter = a.nframes * (a.tiles + a.chunks);
  const long total = (long)per_iter * a.iters;
  const size_t img = (size_t)N * a.nx;
  const PState& g = a.st;

  for (;;) {
    __syncthreads();  // previous item fully done with shared memory and s_*; s_ticket is this item's
    const long t = s_ticket;
    if (t >= total) break;
    int k, f, piece;
    bool normal;
    if (a.lag >= 0) {
      const StaggeredItem it = staggered_item(t, a.nframes * a.iters, a.tiles, a.chunks, a.lag);
      normal = !it.second;
      k = it.unit / a.nframes;
      f = it.unit - k * a.nframes;
      piece = it.piece;
    } else {
      k = (int)(t / per_iter);
      int w = (int)(t - (long)k * per_iter);
      normal = w < a.nframes * a.tiles;
      if (!normal) w -= a.nframes * a.tiles;
      const int per = normal ? a.tiles : a.chunks;
      f = w / per;
      piece = w - f * per;
    }
    const PFrame fr = a.frames[f];
    const int gi = fr.g0;  // this frame's group: state index and first table entry

    // ---- wait for the previous phase of this frame's group ----
    if (threadIdx.x == 0) {
      bool ok = true;
      if (normal) {
        if (k > 0) ok = wait_at_least(g.upd_ready + gi, k);
      } else {
        ok = wait_at_least(g.nrm_ready + gi, k + 1);
      }
      if (!ok) atomicOr(a.err, ERR_TIMEOUT);
      s_ok = ok ? 1 : 0;
      s_active = (ok && k + fr.k0 < fr.kmax) ? __ldcg(fr.active) : 0;
    }
    __syncthreads();
    const bool work = s_ok && s_active;

    if (normal) {
      if (work) {
        tile.prefetch(fr, piece, nfill);  // first coil's maps, overlapping the set-up below
        const int kg = k + fr.k0;  // global iteration index of this frame
        NormalTile nt;
        nt.p_src = (kg > 0 && ((kg - 1) & 1) ? fr.p[1] : fr.p[0]);
        nt.p_dst = ((kg & 1) ? fr.p[1] : fr.p[0]);
        nt.r = fr.r;
        nt.q = fr.q;
        nt.S = fr.S;
        nt.nx = a.nx;
        nt.coils = fr.coils;
        nt.tile = piece;
        nt.p_update = kg > 0 ? 1 : 0;
        nt.centred = 0;
        nt.lambda = fr.lambda;
        nt.lambda_t = fr.lambda_t;
        if (fr.lambda_t != 0.f) {  // neighbours' table entries only for frames coupled in time
          const int ip = kg > 0 ? ((kg - 1) & 1) : 0;
          const PFrame* fp = a.frames + fr.nb_prev;
          const PFrame* fn = a.frames + fr.nb_next;
          nt.r_prev = fp->r;
          nt.ps_prev = ip ? fp->p[1] : fp->p[0];
          nt.r_next = fn->r;
          nt.ps_next = ip ? fn->p[1] : fn->p[0];
        }
        nt.beta = kg > 0 ? (float)__ldcg(fr.beta) : 0.f;
        const float part = tile.run(nt, fr.lines, fr.L, nfill, a.err);
        nfill += (unsigned)fr.coils;
        const double tot = block_sum<T>((double)part, tile.red());
        if (threadIdx.x == 0) __stcg(g.part_nrm + (size_t)f * a.tiles + piece, tot);
      }
      __threadfence();
      if (threadIdx.x == TK) s_ticket = (int)atomicAdd(a.ticket, 1u);  // every thread has read this item's
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(g.nrm_arrive + gi, 1u);
        if (prev == (unsigned)(a.tiles * fr.gsize) - 1u) {  // last tile of the group: alpha
          g.nrm_arrive[gi] = 0u;
          __threadfence();
          if (s_active) {
            double pq = 0.0;
            for (int i = 0; i < a.tiles * fr.gsize; ++i) pq += __ldcg(g.part_nrm + (size_t)gi * a.tiles + i);
            if (pq > 0.0) {
              __stcg(fr.alpha, __ldcg(fr.rho) / pq);
            } else {  // breakdown (zero, negative or NaN curvature): freeze the frame
              __stcg(fr.active, 0);
              __stcg(fr.outcome, CG_BREAKDOWN);
            }
          }
          __threadfence();
          st_release(g.nrm_ready + gi, k + 1);
        }
      }
    } else {
      float acc = 0.f;
      if (work) {
        const float al = (float)__ldcg(fr.alpha);
        const float4* pp = reinterpret_cast<const float4*>((((k + fr.k0) & 1) ? fr.p[1] : fr.p[0]));
        const float4* qp = reinterpret_cast<const float4*>(fr.q);
        float4* xp = reinterpret_cast<float4*>(fr.x);
        float4* rp = reinterpret_cast<float4*>(fr.r);
        const long img4 = (long)(img / 2);
        constexpr int VEC = kUpdateVec;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 1
        for (int rd = 0; rd < kUpdateRounds; ++rd) {
          const long base = ((long)piece * kUpdateRounds + rd) * (T * VEC) + threadIdx.x;
          float4 xv[VEC], pv[VEC], qv[VEC], rv[VEC];
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            const long i = base + j * T;
            const bool ok = i < img4;
            xv[j] = ok ? __ldcg(xp + i) : z;
            pv[j] = ok ? __ldcg(pp + i) : z;
            qv[j] = ok ? __ldcg(qp + i) : z;
            rv[j] = ok ? __ldcg(rp + i) : z;
          }
#pragma unroll
          for (int j = 0; j < VEC; ++j) {
            const long i = base + j * T;
            float4 xn = xv[j], rn = rv[j];
            xn.x = fmaf(al, pv[j].x, xn.x); xn.y = fmaf(al, pv[j].y, xn.y);
            xn.z = fmaf(al, pv[j].z, xn.z); xn.w = fmaf(al, pv[j].w, xn.w);
            rn.x = fmaf(-al, qv[j].x, rn.x); rn.y = fmaf(-al, qv[j].y, rn.y);
            rn.z = fmaf(-al, qv[j].z, rn.z); rn.w = fmaf(-al, qv[j].w, rn.w);
            if (i < img4) {
              __stcg(xp + i, xn);
              __stcg(rp + i, rn);
              acc = fmaf(rn.x, rn.x, fmaf(rn.y, rn.y, fmaf(rn.z, rn.z, fmaf(rn.w, rn.w, acc))));
            }
          }
        }
        const double tot = block_sum<T>((double)acc, tile.red());
        if (threadIdx.x == 0) __stcg(g.part_upd + (size_t)f * a.chunks + piece, tot);
      }
      __threadfence();
      if (threadIdx.x == TK) s_ticket = (int)atomicAdd(a.ticket, 1u);
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(g.upd_arrive + gi, 1u);
        if (prev == (unsigned)(a.chunks * fr.gsize) - 1u) {  // last chunk of the group: beta, stopping test
          g.upd_arrive[gi] = 0u;
          __threadfence();
          if (s_active) {
            double rho_new = 0.0;
            for (int i = 0; i < a.chunks * fr.gsize; ++i) rho_new += __ldcg(g.part_upd + (size_t)gi * a.chunks + i);
            const double rho0 = __ldcg(fr.rho0);
            __stcg(fr.iters, __ldcg(fr.iters) + 1);
            __stcg(fr.resid, sqrt(rho_new / rho0));
            const bool stop = (rho_new == 0.0) || (fr.tol > 0.0 && sqrt(rho_new / rho0) <= fr.tol);
            if (stop) {
              __stcg(fr.active, 0);
              __stcg(fr.outcome, CG_CONVERGED);
            } else {
              __stcg(fr.beta, rho_new / __ldcg(fr.rho));
            }
            __stcg(fr.rho, rho_new);
          }
          __threadfence();
          st_release(g.upd_ready + gi, k + 1);
        }
      }
    }
  }
}

}  // namespace sense
