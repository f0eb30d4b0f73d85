// Uneven batching: CG-SENSE for many instances of different matrix size,
// coil count, frame count and acceleration in one persistent launch per size
// class.
//
// The batch keeps one plan per instance (its workspace and per-frame CG
// state).  Instances are grouped by (ny, nx, storage); the frames of a class
// form one frame table of the persistent CG kernel, so every iteration of
// every frame of the class runs in a single launch whose blocks pipeline
// across instances and frames.  The whole solve -- CG start of every
// instance, one persistent launch per class, the per-instance outputs -- is
// captured once per argument set into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "fused.cuh"
#include "launch.h"
#include "plan.h"
#include "trace.h"
#include "sense.h"

using namespace sense;

struct sense_batch {
  struct Class {
    int ny = 0, nx = 0, storage = 0;
    std::vector<int> members;  // instance indices
    int frames = 0;
    int variant = 0, tiles = 0, chunks = 0;
    int order = kOrderIterationMajor;  // item order its frame table allows (persistent_order)
    int* ints = nullptr;        // nrm_arrive, upd_arrive, nrm_ready, upd_ready ([4][frames]), ticket
    double* part_nrm = nullptr; // [frames][tiles]
    double* part_upd = nullptr; // [frames][chunks]
    size_t part_upd_cap = 0;    // capacity of part_upd per frame
  };
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    std::vector<PFrame*> tables;  // one device frame table per class
  };
  int device = 0;
  int sms = 0;
  std::vector<sense_plan*> plans;
  std::vector<Class> classes;
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  cudaStream_t capture_stream = nullptr;
  std::map<std::vector<const void*>, Graph> graphs;
};

namespace {

sense_status bfail(sense_status st, const std::string& m) {
  record_error(m);
  return st;
}

#define SENSE_BATCH_CUDA(expr)                                                                   \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) return bfail(SENSE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

template <class T>
sense_status balloc(sense_batch* b, T** out, size_t count) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(count * sizeof(T), 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return bfail(SENSE_ENOMEM, "batch workspace allocation failed: " + std::string(cudaGetErrorString(e)));
  }
  b->allocs.push_back(p);
  b->ws_bytes += count * sizeof(T);
  *out = static_cast<T*>(p);
  return SENSE_OK;
}

void drop_graphs(sense_batch* b) {
  for (auto& kv : b->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (PFrame* t : kv.second.tables) cudaFree(t);
  }
  b->graphs.clear();
}

void batch_release(sense_batch* b) {
  drop_graphs(b);
  for (sense_plan* p : b->plans)
    if (p) sense_plan_destroy(p);
  b->plans.clear();
  for (void* p : b->allocs) cudaFree(p);
  b->allocs.clear();
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  b->capture_stream = nullptr;
}

// Tile and chunk counts of a class for its variant (the persistent kernel's
// partition of a frame).
void class_partition(sense_batch::Class& c) {
  const int W = normal_variant_width(c.ny, c.variant);
  const int th = normal_variant_threads(c.ny, c.variant);
  c.tiles = (c.nx + W - 1) / W;
  c.chunks = update_chunks((size_t)c.ny * c.nx, th);
}

sense_status run_batch(sense_batch* b, const sense_batch_io* io, const std::vector<PFrame*>& tables, int max_iter,
                       double tol, cudaStream_t st) {
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    sense_batch::Class& c = b->classes[ci];
    for (int i : c.members) {
      sense_status rc = plan_cg_start(b->plans[i], io[i].y, io[i].S, io[i].lines,
                                      reinterpret_cast<float2*>(io[i].x_out), tol, st);
      const void* maps = nullptr;  // refresh S^T (its buffer exists) for lane-major variants
      if (rc == SENSE_OK) rc = plan_maps(b->plans[i], io[i].S, st, &maps);
      if (rc != SENSE_OK) return rc;
    }
    if (max_iter > 0) {
      SENSE_BATCH_CUDA(cudaMemsetAsync(c.ints, 0, sizeof(int) * (4 * (size_t)c.frames + 1), st));
      PArgs a{};
      a.frames = tables[ci];
      a.nframes = c.frames;
      a.nx = c.nx;
      a.tiles = c.tiles;
      a.chunks = c.chunks;
      a.lag = c.order;
      a.iters = max_iter;
      a.ticket = reinterpret_cast<unsigned*>(c.ints + 4 * c.frames);
      a.tw = b->plans[c.members[0]]->tw_y;
      a.err = b->plans[c.members[0]]->err();
      a.st.nrm_arrive = reinterpret_cast<unsigned*>(c.ints);
      a.st.upd_arrive = reinterpret_cast<unsigned*>(c.ints + c.frames);
      a.st.nrm_ready = c.ints + 2 * c.frames;
      a.st.upd_ready = c.ints + 3 * c.frames;
      a.st.part_nrm = c.part_nrm;
      a.st.part_upd = c.part_upd;
      cudaError_t e = c.storage == SENSE_STORE_BF16
                          ? launch_cg_persistent<StBF16>(c.ny, c.variant, a, b->sms, st)
                          : launch_cg_persistent<StC64>(c.ny, c.variant, a, b->sms, st);
      if (e != cudaSuccess) return bfail(SENSE_ECUDA, std::string("persistent CG (batch): ") + cudaGetErrorString(e));
    }
    for (int i : c.members) {
      sense_status rc = plan_centred_output(b->plans[i], reinterpret_cast<float2*>(io[i].x_out), st);
      if (rc == SENSE_OK)
        rc = plan_cg_finish(b->plans[i], io[i].iters_out, io[i].rel_resid_out, io[i].outcome_out, st);
      if (rc != SENSE_OK) return rc;
    }
  }
  return SENSE_OK;
}

}  // namespace

extern "C" {

sense_status sense_batch_create(const sense_shape* shapes, int count, int device, sense_batch** out) {
  sense::TraceRange trace_range("sense_batch_create");
  if (!out || !shapes || count < 1) return bfail(SENSE_EINVAL, "need shapes, count >= 1 and out");
  *out = nullptr;
  int ndev = 0;
  SENSE_BATCH_CUDA(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return bfail(SENSE_EINVAL, "device index out of range");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  sense_batch* b = new sense_batch();
  b->device = device;
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, device);
  sense_status rc = SENSE_OK;
  b->plans.assign(count, nullptr);
  for (int i = 0; i < count && rc == SENSE_OK; ++i) {
    rc = sense_plan_create(&shapes[i], device, &b->plans[i]);
    if (rc == SENSE_OK) sense_plan_set_cg_mode(b->plans[i], 1);
  }
  if (rc == SENSE_OK) {
    std::map<std::tuple<int, int, int>, int> index;
    for (int i = 0; i < count; ++i) {
      auto key = std::make_tuple(shapes[i].ny, shapes[i].nx, shapes[i].storage);
      auto it = index.find(key);
      if (it == index.end()) {
        sense_batch::Class c;
        c.ny = shapes[i].ny;
        c.nx = shapes[i].nx;
        c.storage = shapes[i].storage;
        it = index.emplace(key, (int)b->classes.size()).first;
        b->classes.push_back(c);
      }
      sense_batch::Class& c = b->classes[it->second];
      c.members.push_back(i);
      c.frames += shapes[i].frames;
    }
    for (auto& c : b->classes) {
      class_partition(c);
      // room for the narrowest tiles and the smallest blocks of any variant
      int min_threads = 1 << 30;
      for (int v = 0; v < kNormVariants; ++v) {
        const int th = normal_variant_threads(c.ny, v);
        if (th > 0) min_threads = std::min(min_threads, th);
      }
      c.part_upd_cap = (size_t)update_chunks((size_t)c.ny * c.nx, min_threads);
      if ((rc = balloc(b, &c.ints, 4 * (size_t)c.frames + 1)) != SENSE_OK) break;
      if ((rc = balloc(b, &c.part_nrm, (size_t)c.frames * ((c.nx + 3) / 4))) != SENSE_OK) break;
      if ((rc = balloc(b, &c.part_upd, (size_t)c.frames * c.part_upd_cap)) != SENSE_OK) break;
    }
  }
  if (rc == SENSE_OK) {
    cudaError_t e = cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) rc = bfail(SENSE_ECUDA, "batch stream: " + std::string(cudaGetErrorString(e)));
  }
  if (rc != SENSE_OK) {
    batch_release(b);
    delete b;
    cudaSetDevice(prev);
    return rc;
  }
  cudaSetDevice(prev);
  *out = b;
  return SENSE_OK;
}

sense_status sense_batch_destroy(sense_batch* b) {
  if (!b) return SENSE_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  batch_release(b);
  delete b;
  cudaSetDevice(prev);
  return SENSE_OK;
}

size_t sense_batch_workspace_bytes(const sense_batch* b) {
  if (!b) return 0;
  size_t s = b->ws_bytes;
  for (const sense_plan* p : b->plans) s += sense_plan_workspace_bytes(p);
  return s;
}

int sense_batch_classes(const sense_batch* b) { return b ? (int)b->classes.size() : 0; }

sense_status sense_batch_autotune(sense_batch* b, const sense_batch_io* io, void* stream) {
  sense::TraceRange trace_range("sense_batch_autotune");
  if (!b || !io) return bfail(SENSE_EINVAL, "batch and io are required");
  for (auto& c : b->classes) {
    // representative: the member with the most frames
    int rep = c.members[0];
    for (int i : c.members)
      if (b->plans[i]->sh.frames > b->plans[rep]->sh.frames) rep = i;
    int v = 0;
    sense_status rc = sense_plan_autotune(b->plans[rep], io[rep].S, io[rep].lines, &v, nullptr, stream);
    if (rc != SENSE_OK) return rc;
    c.variant = v;
    for (int i : c.members) {
      rc = sense_plan_set_variant(b->plans[i], v);
      if (rc != SENSE_OK) return rc;
    }
    class_partition(c);
  }
  drop_graphs(b);
  return SENSE_OK;
}

sense_status sense_batch_set_lambda(sense_batch* b, int instance, double lambda) {
  if (!b) return bfail(SENSE_EINVAL, "batch is NULL");
  if (instance < 0 || instance >= (int)b->plans.size()) return bfail(SENSE_EINVAL, "instance index out of range");
  sense_status rc = sense_plan_set_lambda(b->plans[instance], lambda);
  if (rc != SENSE_OK) return rc;
  drop_graphs(b);  // frame tables bake lambda in
  return SENSE_OK;
}

sense_status sense_batch_set_temporal(sense_batch* b, int instance, double lambda_t) {
  if (!b) return bfail(SENSE_EINVAL, "batch is NULL");
  if (instance < 0 || instance >= (int)b->plans.size()) return bfail(SENSE_EINVAL, "instance index out of range");
  sense_status rc = sense_plan_set_temporal(b->plans[instance], lambda_t);
  if (rc != SENSE_OK) return rc;
  drop_graphs(b);  // frame tables bake the coupling in
  return SENSE_OK;
}

sense_status sense_batch_set_variant(sense_batch* b, int ny, int variant) {
  if (!b) return bfail(SENSE_EINVAL, "batch is NULL");
  for (auto& c : b->classes) {
    if (c.ny != ny) continue;
    if (normal_variant_width(ny, variant) <= 0) return bfail(SENSE_EINVAL, "no such variant");
    c.variant = variant;
    for (int i : c.members) {
      sense_status rc = sense_plan_set_variant(b->plans[i], variant);
      if (rc != SENSE_OK) return rc;
    }
    class_partition(c);
  }
  drop_graphs(b);
  return SENSE_OK;
}

sense_status sense_batch_cg_solve(sense_batch* b, const sense_batch_io* io, int max_iter, double rel_tol,
                                  void* stream) {
  sense::TraceRange trace_range("sense_batch_cg_solve");
  if (!b || !io) return bfail(SENSE_EINVAL, "batch and io are required");
  if (max_iter < 0 || !(rel_tol >= 0.0)) return bfail(SENSE_EINVAL, "max_iter must be >= 0 and rel_tol >= 0");
  const int count = (int)b->plans.size();
  std::vector<const void*> key;
  key.reserve(7 * (size_t)count + 2);
  for (int i = 0; i < count; ++i) {
    const sense_batch_io& o = io[i];
    auto a16 = [](const void* p) { return p && ((reinterpret_cast<uintptr_t>(p) & 15u) == 0); };
    if (!a16(o.y) || !a16(o.S) || !a16(o.x_out) || !o.lines || (reinterpret_cast<uintptr_t>(o.lines) & 3u))
      return bfail(SENSE_EINVAL, "instance " + std::to_string(i) + ": y, S, x_out 16-byte aligned, lines 4-byte");
    key.insert(key.end(), {o.y, o.S, (const void*)o.lines, (const void*)o.x_out, (const void*)o.iters_out,
                           (const void*)o.rel_resid_out, (const void*)o.outcome_out});
  }
  key.push_back(reinterpret_cast<const void*>((intptr_t)max_iter));
  double tol_copy = rel_tol;
  const void* tol_bits = nullptr;
  static_assert(sizeof(double) == sizeof(void*), "pointer-sized double");
  memcpy(&tol_bits, &tol_copy, sizeof(double));
  key.push_back(tol_bits);

  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  auto it = b->graphs.find(key);
  if (it == b->graphs.end()) {
    if (b->graphs.size() >= 8) drop_graphs(b);
    sense_batch::Graph g;
    // frame tables of this argument set (device copies, uploaded now)
    for (auto& c : b->classes) {
      std::vector<PFrame> host((size_t)c.frames);
      size_t off = 0;
      for (int i : c.members) {
        sense_plan* p = b->plans[i];
        const bool transposed = plan_maps_transposed(p);
        sense_status trc = transposed ? plan_maps_buffer(p) : plan_prepare_tmap(p, io[i].S, st);
        if (trc != SENSE_OK) {
          for (PFrame* t : g.tables) cudaFree(t);
          cudaSetDevice(prev);
          return trc;
        }
        plan_frames(p, transposed ? p->maps_t : io[i].S, io[i].lines, reinterpret_cast<float2*>(io[i].x_out), 0,
                    rel_tol, host.data() + off, (int)off);
        off += p->sh.frames;
      }
      PFrame* dev = nullptr;
      cudaError_t e = cudaMalloc(&dev, sizeof(PFrame) * host.size());
      if (e == cudaSuccess) e = cudaMemcpy(dev, host.data(), sizeof(PFrame) * host.size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        if (dev) cudaFree(dev);
        for (PFrame* t : g.tables) cudaFree(t);
        cudaSetDevice(prev);
        return bfail(SENSE_ECUDA, std::string("batch frame table: ") + cudaGetErrorString(e));
      }
      g.tables.push_back(dev);
      c.order = persistent_order(host.data(), c.frames);
    }
    // kernel attributes are set outside the capture (empty grids launch nothing)
    for (auto& c : b->classes) {
      PArgs none{};
      CUtensorMap none_map{};  // no work below: the launchers only set kernel attributes
      const FusedSched none_sched{nullptr, nullptr, 0, 0, 0, 1};
      if (c.storage == SENSE_STORE_BF16) {
        RowArgs<__nv_bfloat162, float2> ra{};
        AdjColArgs<StBF16> aa{};
        launch_rows_inv<StBF16>(c.nx, ra, st);
        launch_adj_col<StBF16>(c.ny, 1, aa, 0, 0, st);
        launch_adj_col_tma<StBF16>(c.ny, 1, none_map, none_map, aa, 0, b->sms, st);
        launch_adjoint_fused<StBF16>(c.ny, 1, true, none_map, none_map, aa, nullptr, nullptr, none_sched, 1.f, b->sms, st);
      } else {
        RowArgs<float2, float2> ra{};
        AdjColArgs<StC64> aa{};
        launch_rows_inv<StC64>(c.nx, ra, st);
        launch_adj_col<StC64>(c.ny, 1, aa, 0, 0, st);
        launch_adj_col_tma<StC64>(c.ny, 1, none_map, none_map, aa, 0, b->sms, st);
        launch_adjoint_fused<StC64>(c.ny, 1, false, none_map, none_map, aa, nullptr, nullptr, none_sched, 1.f, b->sms, st);
      }
      cudaError_t e = c.storage == SENSE_STORE_BF16 ? launch_cg_persistent<StBF16>(c.ny, c.variant, none, b->sms, st)
                                                    : launch_cg_persistent<StC64>(c.ny, c.variant, none, b->sms, st);
      if (e != cudaSuccess) {
        for (PFrame* t : g.tables) cudaFree(t);
        cudaSetDevice(prev);
        return bfail(SENSE_ECUDA, std::string("persistent kernel set-up: ") + cudaGetErrorString(e));
      }
    }
    cudaStream_t cs = b->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sense_status rc = e == cudaSuccess ? run_batch(b, io, g.tables, max_iter, rel_tol, cs)
                                       : bfail(SENSE_ECUDA, "begin capture failed");
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(cs, &graph);
    if (rc == SENSE_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != SENSE_OK || e != cudaSuccess) {
      for (PFrame* t : g.tables) cudaFree(t);
      cudaSetDevice(prev);
      return rc != SENSE_OK ? rc : bfail(SENSE_ECUDA, std::string("batch graph: ") + cudaGetErrorString(e));
    }
    it = b->graphs.emplace(key, g).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second.exec, st);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return bfail(SENSE_ECUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
  return SENSE_OK;
}

sense_status sense_batch_check(sense_batch* b, void* stream) {
  sense::TraceRange trace_range("sense_batch_check");
  if (!b) return bfail(SENSE_EINVAL, "batch is NULL");
  for (sense_plan* p : b->plans) {
    sense_status rc = sense_plan_check(p, stream);
    if (rc != SENSE_OK) return rc;
  }
  return SENSE_OK;
}

}  // extern "C"
