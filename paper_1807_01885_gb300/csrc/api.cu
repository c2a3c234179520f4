// C ABI of libbem.so (declared in include/bem.h): argument checks, workspace
// ownership, host/device argument staging, error reporting.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <vector>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "bem_internal.cuh"

namespace bem {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void note_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_last_error = msg; }

bem_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? BEM_ENOMEM : BEM_ECUDA;
}

bem_status solve_contact_device(bem_kernel_s* k, const bem_problem* prob, const void* f, const void* pinit,
                                uint8_t* mask, void* p_out, bem_result* res, cudaStream_t s);
bem_status solve_batch_device(int n, bem_kernel_s* const* ks, const bem_problem* probs, const bool* has_pinit,
                              bem_result* res, cudaStream_t const* strm);
void release_batch_graph(const bem_kernel_s* k);

// Argument checks of an operator description (shared with the allocation-free
// entry point).
bem_status check_desc(const bem_kernel_desc* d) {
  if (d == nullptr) { set_error("desc is NULL"); return BEM_EINVAL; }
  const int N = d->N;
  if (N < 4 || N > (1 << MAX_LOGN) || (N & (N - 1))) {
    set_error("N must be a power of two in [4, 2048]");
    return BEM_EINVAL;
  }
  if (d->precision != BEM_FP64 && d->precision != BEM_FP32) { set_error("unknown precision"); return BEM_EINVAL; }
  if (d->dc_mode != BEM_DC_FINITE_PART && d->dc_mode != BEM_DC_ZERO) { set_error("unknown dc_mode"); return BEM_EINVAL; }
  if (!(d->delta > 0.0) || !isfinite(d->delta)) { set_error("delta must be positive and finite"); return BEM_EINVAL; }
  if (!(d->h >= 0.0) || isnan(d->h)) { set_error("h must be >= 0 (INFINITY allowed)"); return BEM_EINVAL; }
  if (!(d->E1 > 0.0) || !isfinite(d->E1)) { set_error("E1 must be positive and finite"); return BEM_EINVAL; }
  if (!(d->E2 > 0.0) || isnan(d->E2)) { set_error("E2 must be positive (INFINITY allowed)"); return BEM_EINVAL; }
  if (!(d->nu1 >= 0.0 && d->nu1 < 0.5) || !(d->nu2 >= 0.0 && d->nu2 < 0.5)) {
    set_error("Poisson ratios must lie in [0, 0.5)");
    return BEM_EINVAL;
  }
  if (d->op_kind != BEM_OP_PERIODIC && d->op_kind != BEM_OP_OPEN) { set_error("unknown op_kind"); return BEM_EINVAL; }
  if (d->op_kind == BEM_OP_OPEN && !open_plane_homogeneous(*d)) {
    set_error("the open-plane operator is built for a homogeneous half-space (h = INFINITY, h = 0 or equal "
              "materials)");
    return BEM_EUNSUPPORTED;
  }
  return BEM_OK;
}

namespace {

// NVTX range around an entry point (shown by Nsight tools; no cost when none attaches)
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

bem_status check_problem(const bem_problem* prob) {
  if (prob == nullptr || prob->height == nullptr) {
    set_error("NULL problem or height map");
    return BEM_EINVAL;
  }
  if (!(prob->tol > 0.0) || prob->max_iter <= 0 || !(prob->dgamma >= 0.0) || !isfinite(prob->target)) {
    set_error("invalid problem (tol > 0, max_iter > 0, dgamma >= 0, finite target)");
    return BEM_EINVAL;
  }
  if (prob->control != BEM_CTRL_DEPTH && prob->control != BEM_CTRL_FORCE) {
    set_error("unknown control");
    return BEM_EINVAL;
  }
  if (prob->control == BEM_CTRL_FORCE && prob->dgamma == 0.0 && !(prob->target > 0.0)) {
    set_error("non-adhesive force control needs a positive force");
    return BEM_EINVAL;
  }
  return BEM_OK;
}

// Library-owned non-blocking streams for concurrent batch instances (per device).
constexpr int kBatchStreams = 32;
cudaStream_t batch_stream(int dev, int i) {
  static std::mutex mu;
  static std::vector<std::vector<cudaStream_t>> pools;
  std::lock_guard<std::mutex> lock(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1);
  auto& pool = pools[dev];
  if (pool.empty()) {
    pool.resize(kBatchStreams, nullptr);
    for (auto& st : pool) cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  }
  return pool[i % kBatchStreams];
}

}  // namespace

cudaStream_t capture_stream() {
  static std::mutex mu;
  static std::vector<cudaStream_t> per_dev;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  if ((int)per_dev.size() <= dev) per_dev.resize(dev + 1, nullptr);
  if (per_dev[dev] == nullptr) cudaStreamCreateWithFlags(&per_dev[dev], cudaStreamNonBlocking);
  return per_dev[dev];
}

uint64_t next_serial() {
  static std::atomic<uint64_t> ctr{0};
  return ++ctr;
}

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// A workspace array with guard zones on both sides (see kGuard).
template <typename P>
cudaError_t alloc_guarded(Workspace& w, P** p, size_t bytes) {
  if (w.n_guards >= kMaxGuarded) return cudaErrorInvalidValue;
  unsigned char* base = nullptr;
  cudaError_t e = cudaMalloc((void**)&base, bytes + 2 * kGuard);
  if (e != cudaSuccess) return e;
  if ((e = cudaMemset(base, kGuardByte, kGuard)) != cudaSuccess ||
      (e = cudaMemset(base + kGuard + bytes, kGuardByte, kGuard)) != cudaSuccess) {
    cudaFree(base);
    return e;
  }
  w.guards[w.n_guards++] = GuardRec{base, bytes};
  *p = reinterpret_cast<P*>(base + kGuard);
  return cudaSuccess;
}

__global__ void k_guard_scan(const unsigned char* __restrict__ lead, const unsigned char* __restrict__ trail,
                             unsigned long long* bad) {
  const unsigned i = threadIdx.x;   // one thread per guard byte pair
  unsigned n = 0;
  if (i < kGuard) n = (lead[i] != kGuardByte) + (trail[i] != kGuardByte);
  if (n) atomicAdd(bad, (unsigned long long)n);
}

void free_ws(bem_kernel_s* k) {
  Workspace& w = k->ws;
  for (int i = 0; i < w.n_guards; ++i) cudaFree(w.guards[i].base);
  cudaFree(w.guard_bad);
  cudaFree(w.ticket);
  cudaFree(w.state);
  cudaFreeHost(w.state_host);
  cudaFreeHost(w.aux_host);
  if (w.done_ev != nullptr) cudaEventDestroy(w.done_ev);
  w = Workspace{};
}

// Host <-> device staging of an N*N array argument.
struct Arg {
  const void* dev = nullptr;
  bool host = false;
};

bem_status stage_in(bem_kernel_s* k, const void* p, void* dst, size_t bytes, cudaStream_t s, Arg* out) {
  if (p == nullptr) { out->dev = nullptr; return BEM_OK; }
  if (is_device_ptr(p)) {
    out->dev = p;
    out->host = false;
    return BEM_OK;
  }
  BEM_CUDA_TRY(cudaMemcpyAsync(dst, p, bytes, cudaMemcpyHostToDevice, s));
  out->dev = dst;
  out->host = true;
  return BEM_OK;
}

}  // namespace
}  // namespace bem

using namespace bem;

extern "C" {

int32_t bem_version(void) { return 100; }

int64_t bem_launch_count(void) { return (int64_t)launches(); }

bem_status bem_profile_passes(bem_kernel k, const void* p, void* u, int32_t reps, float* ms_out,
                              void* cuda_stream) {
  if (k == nullptr || p == nullptr || u == nullptr || ms_out == nullptr || reps <= 0) {
    set_error("invalid profiling arguments");
    return BEM_EINVAL;
  }
  if (!is_device_ptr(p) || !is_device_ptr(u)) {
    set_error("profiling needs device arrays");
    return BEM_EINVAL;
  }
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) BEM_CUDA_TRY(cudaEventCreate(&ev[i]));
  double acc[3] = {0, 0, 0};
  bem_status st = BEM_OK;
  for (int r = 0; r < reps && st == BEM_OK; ++r) {
    cudaEventRecord(ev[0], s);
    for (int pass = 0; pass < 3; ++pass) {
      if (k->prec == BEM_FP64)
        launch_pass<double>(k, pass, (const double*)p, (double*)u, s);
      else
        launch_pass<float>(k, pass, (const float*)p, (float*)u, s);
      cudaEventRecord(ev[pass + 1], s);
    }
    cudaError_t e = cudaEventSynchronize(ev[3]);
    if (e != cudaSuccess) { st = cuda_fail(e, "profile"); break; }
    for (int pass = 0; pass < 3; ++pass) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[pass], ev[pass + 1]);
      acc[pass] += ms;
    }
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  for (int pass = 0; pass < 3; ++pass) ms_out[pass] = (float)(acc[pass] / reps);
  return st;
}

const char* bem_last_error(void) { return g_last_error.c_str(); }

bem_status bem_set_pass_timing(bem_kernel k, int32_t on) {
  if (k == nullptr) { set_error("NULL kernel"); return BEM_EINVAL; }
  k->timing.on = on ? 1 : 0;
  return BEM_OK;
}

bem_status bem_pass_timing(bem_kernel k, double* ms_total, int64_t* launches_out, int32_t reset) {
  if (k == nullptr || ms_total == nullptr || launches_out == nullptr) { set_error("NULL argument"); return BEM_EINVAL; }
  DeviceGuard g(k->dev);
  BEM_CUDA_TRY(cudaDeviceSynchronize());
  harvest_pass_timing(k);
  for (int pass = 0; pass < 3; ++pass) {
    ms_total[pass] = k->timing.ms[pass];
    launches_out[pass] = k->timing.n[pass];
    if (reset) {
      k->timing.ms[pass] = 0.0;
      k->timing.n[pass] = 0;
    }
  }
  return BEM_OK;
}

// ---- radix choice and autotuner ---------------------------------------------
static int cur_row_log2(const bem_kernel_s* k) { return (k->prec == BEM_FP32 && !k->row_radix_alt) ? 4 : 3; }
static int cur_col_log2(const bem_kernel_s* k) { return (k->prec == BEM_FP32 && !k->col_radix_alt) ? 4 : 3; }

// Sets the radix flags, rebuilds the stage twiddles and drops the captured CG graph
// (it holds launches of the previous kernels).  Asynchronous on s.
static bem_status apply_radix(bem_kernel_s* k, int row_log2, int col_log2, cudaStream_t s) {
  const bool f32 = k->prec == BEM_FP32;
  k->row_radix_alt = (f32 && row_log2 == 3) ? 1 : 0;
  k->col_radix_alt = (f32 && col_log2 == 3) ? 1 : 0;
  if (f32) reg_twiddles<float>(k, s);
  else reg_twiddles<double>(k, s);
  note_launches(2);
  BEM_CUDA_TRY(cudaGetLastError());
  if (k->graphs.pk_exec != nullptr) {
    BEM_CUDA_TRY(cudaGraphExecDestroy(k->graphs.pk_exec));
    k->graphs.pk_exec = nullptr;
    k->graphs.pk_nodes = 0;
  }
  if (k->graphs.lin_exec != nullptr) {
    BEM_CUDA_TRY(cudaGraphExecDestroy(k->graphs.lin_exec));
    k->graphs.lin_exec = nullptr;
    k->graphs.lin_nodes = 0;
  }
  if (k->graphs.loop_exec != nullptr) {
    BEM_CUDA_TRY(cudaGraphExecDestroy(k->graphs.loop_exec));
    k->graphs.loop_exec = nullptr;
    k->graphs.loop_nodes = 0;
  }
  k->serial = next_serial();
  k->graphs.warm = 0;   // the next chunk runs plainly once (attributes of the new kernels)
  k->graphs.lin_warm = 0;
  return BEM_OK;
}

static bool radix_allowed(const bem_kernel_s* k, int v) { return v == 3 || (k->prec == BEM_FP32 && v == 4); }

bem_status bem_set_radix(bem_kernel k, int32_t row_log2_radix, int32_t col_log2_radix, void* cuda_stream) {
  if (k == nullptr) { set_error("NULL kernel"); return BEM_EINVAL; }
  if (!radix_allowed(k, row_log2_radix) || !radix_allowed(k, col_log2_radix)) {
    set_error("log2 radix must be 3 (or 4 on the float path)");
    return BEM_EINVAL;
  }
  if (k->logN < 4) return BEM_OK;
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  bem_status st = apply_radix(k, row_log2_radix, col_log2_radix, s);
  if (st != BEM_OK) return st;
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_autotune(bem_kernel k, int32_t reps, int32_t* choice_out, void* cuda_stream) {
  if (k == nullptr || reps <= 0) { set_error("invalid autotune arguments"); return BEM_EINVAL; }
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int best_row = cur_row_log2(k), best_col = cur_col_log2(k);
  if (k->logN >= 4 && k->prec == BEM_FP32) {
    // input and output of the timed passes: two of the handle's solver vectors
    const size_t n = (size_t)k->N * k->N;
    float* pin = (float*)k->ws.vec + 6 * n;
    float* uout = (float*)k->ws.vec + 4 * n;
    BEM_CUDA_TRY(cudaMemsetAsync(pin, 0x3f, n * sizeof(float), s));   // finite values (0.747...)
    cudaEvent_t e0, e1;
    BEM_CUDA_TRY(cudaEventCreate(&e0));
    BEM_CUDA_TRY(cudaEventCreate(&e1));
    // minimum time over reps of the row passes (0 and 2) or the column pass (1),
    // after two untimed launches
    auto time_passes = [&](bool rows) -> float {
      float best = 1e30f;
      for (int r = 0; r < reps + 2; ++r) {
        cudaEventRecord(e0, s);
        if (rows) {
          launch_pass<float>(k, 0, pin, uout, s);
          launch_pass<float>(k, 2, pin, uout, s);
        } else {
          launch_pass<float>(k, 1, pin, uout, s);
        }
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r >= 2 && ms < best) best = ms;
      }
      return best;
    };
    bem_status st = BEM_OK;
    float t_best = 1e30f;
    for (int cand : {4, 3}) {   // rows: forward and inverse passes together
      if ((st = apply_radix(k, cand, best_col, s)) != BEM_OK) break;
      const float t = time_passes(true);
      if (t < t_best) { t_best = t; best_row = cand; }
    }
    t_best = 1e30f;
    for (int cand : {4, 3}) {   // columns
      if (st != BEM_OK) break;
      if ((st = apply_radix(k, best_row, cand, s)) != BEM_OK) break;
      const float t = time_passes(false);
      if (t < t_best) { t_best = t; best_col = cand; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != BEM_OK) return st;
    BEM_CUDA_TRY(cudaGetLastError());
    if ((st = apply_radix(k, best_row, best_col, s)) != BEM_OK) return st;
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (choice_out != nullptr) {
    choice_out[0] = best_row;
    choice_out[1] = best_col;
  }
  return BEM_OK;
}

static bem_status make_kernel(const bem_kernel_desc* desc, int32_t n_layers, const bem_layer* layers,
                              void* cuda_stream, bem_kernel* out) {
  if (out == nullptr) { set_error("out is NULL"); return BEM_EINVAL; }
  *out = nullptr;
  bem_kernel_desc dd;
  if (n_layers > 0) {
    if (desc == nullptr || layers == nullptr) { set_error("NULL desc or layer list"); return BEM_EINVAL; }
    if (n_layers > BEM_MAX_LAYERS) { set_error("at most BEM_MAX_LAYERS layers"); return BEM_EINVAL; }
    double H = 0.0;
    for (int l = 0; l < n_layers; ++l) {
      const bem_layer& L = layers[l];
      if (!(L.h >= 0.0) || !isfinite(L.h) || !(L.E > 0.0) || !isfinite(L.E) || !(L.nu >= 0.0 && L.nu < 0.5)) {
        set_error("layer " + std::to_string(l) + ": needs 0 <= h < inf, 0 < E < inf, 0 <= nu < 0.5");
        return BEM_EINVAL;
      }
      H += L.h;
    }
    if (!(H > 0.0)) { set_error("the layer stack needs a positive total thickness"); return BEM_EINVAL; }
    dd = *desc;
    dd.h = H;
    dd.E1 = layers[0].E;
    dd.nu1 = layers[0].nu;
    desc = &dd;
  } else if (n_layers < 0) {
    set_error("negative layer count");
    return BEM_EINVAL;
  }
  bem_status st = check_desc(desc);
  if (st != BEM_OK) return st;
  if (n_layers > 0 && desc->op_kind == BEM_OP_OPEN) {
    set_error("the open-plane operator is built for a homogeneous half-space, not a coating stack");
    return BEM_EUNSUPPORTED;
  }
  bem_kernel_s* k = new bem_kernel_s();
  k->desc = *desc;
  k->n_layers = n_layers;
  for (int l = 0; l < n_layers; ++l) k->layers[l] = layers[l];
  k->serial = next_serial();
  k->N = desc->N;
  k->M = 2 * desc->N;
  k->logN = 0;
  while ((1 << k->logN) < k->N) ++k->logN;
  k->prec = desc->precision;
  k->elem = (k->prec == BEM_FP64) ? sizeof(double) : sizeof(float);
  cudaGetDevice(&k->dev);
  // radix 16 for every float pass until bem_set_radix or bem_autotune says otherwise
  k->col_radix_alt = 0;
  k->row_radix_alt = 0;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)k->N * k->N;
  Workspace& w = k->ws;
  auto fail = [&](cudaError_t e, const char* what) {
    bem_status r = cuda_fail(e, what);
    free_ws(k);
    delete k;
    return r;
  };
  cudaError_t e;
  if ((e = alloc_guarded(w, &w.spec, spec_bytes(k))) != cudaSuccess) return fail(e, "cudaMalloc(spec)");
  if ((e = alloc_guarded(w, &w.table, table_bytes(k))) != cudaSuccess) return fail(e, "cudaMalloc(table)");
  if ((e = alloc_guarded(w, &w.table64, (size_t)(k->N + 1) * (k->N + 1) * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMalloc(table64)");
  if ((e = alloc_guarded(w, &w.tw, (size_t)k->M * 2 * k->elem)) != cudaSuccess) return fail(e, "cudaMalloc(tw)");
  if ((e = alloc_guarded(w, &w.twr, (size_t)stage_tw_count(k->logN) * 2 * k->elem)) != cudaSuccess)
    return fail(e, "cudaMalloc(twr)");
  if ((e = alloc_guarded(w, &w.twc, (size_t)stage_tw_count(k->logN + 1) * 2 * k->elem)) != cudaSuccess)
    return fail(e, "cudaMalloc(twc)");
  if (k->prec == BEM_FP32 &&
      (e = alloc_guarded(w, &w.twpc, (size_t)pair_tw_count(k->logN + 1) * 4 * sizeof(float))) != cudaSuccess)
    return fail(e, "cudaMalloc(twpc)");
  if ((e = alloc_guarded(w, &w.vec, 7 * n * k->elem)) != cudaSuccess) return fail(e, "cudaMalloc(vec)");
  if ((e = alloc_guarded(w, &w.mask, 2 * n)) != cudaSuccess) return fail(e, "cudaMalloc(mask)");
  if ((e = alloc_guarded(w, &w.partials, 16 * 2048 * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMalloc(partials)");
  if ((e = cudaMalloc((void**)&w.ticket, sizeof(unsigned int))) != cudaSuccess) return fail(e, "cudaMalloc(ticket)");
  if ((e = cudaMalloc((void**)&w.guard_bad, sizeof(unsigned long long))) != cudaSuccess)
    return fail(e, "cudaMalloc(guard counter)");
  if ((e = cudaMalloc((void**)&w.state, sizeof(SolveState))) != cudaSuccess) return fail(e, "cudaMalloc(state)");
  if ((e = cudaMallocHost((void**)&w.state_host, sizeof(SolveState))) != cudaSuccess)
    return fail(e, "cudaMallocHost(state)");
  if ((e = cudaMallocHost((void**)&w.aux_host, 16 * sizeof(double))) != cudaSuccess)
    return fail(e, "cudaMallocHost(aux)");
  if ((e = cudaEventCreateWithFlags(&w.done_ev, cudaEventDisableTiming)) != cudaSuccess)
    return fail(e, "cudaEventCreate");
  if ((e = alloc_guarded(w, &w.stage_in, n * k->elem)) != cudaSuccess) return fail(e, "cudaMalloc(stage_in)");
  if ((e = alloc_guarded(w, &w.stage_out, n * k->elem)) != cudaSuccess) return fail(e, "cudaMalloc(stage_out)");
  if ((e = cudaMemsetAsync(w.ticket, 0, sizeof(unsigned int), s)) != cudaSuccess) return fail(e, "memset(ticket)");
  st = build_table(k, s);
  if (st != BEM_OK) {
    free_ws(k);
    delete k;
    return st;
  }
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(e, "build_table");
  *out = k;
  return BEM_OK;
}

bem_status bem_make_kernel(const bem_kernel_desc* desc, void* cuda_stream, bem_kernel* out) {
  Range range("bem_make_kernel");
  return make_kernel(desc, 0, nullptr, cuda_stream, out);
}

bem_status bem_make_kernel_layers(const bem_kernel_desc* desc, int32_t n_layers, const bem_layer* layers,
                                  void* cuda_stream, bem_kernel* out) {
  if (n_layers < 1) {
    if (out != nullptr) *out = nullptr;
    set_error("bem_make_kernel_layers needs 1 <= n_layers <= BEM_MAX_LAYERS");
    return BEM_EINVAL;
  }
  return make_kernel(desc, n_layers, layers, cuda_stream, out);
}

bem_status bem_rebuild_kernel(bem_kernel k, const bem_kernel_desc* desc, void* cuda_stream) {
  if (k == nullptr) { set_error("NULL kernel"); return BEM_EINVAL; }
  bem_status st = check_desc(desc);
  if (st != BEM_OK) return st;
  if (desc->N != k->N || desc->precision != k->prec) {
    set_error("bem_rebuild_kernel: N and precision must equal the handle's");
    return BEM_EINVAL;
  }
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k->desc = *desc;
  k->n_layers = 0;
  st = build_table(k, s);
  if (st != BEM_OK) return st;
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_destroy_kernel(bem_kernel k) {
  if (k == nullptr) return BEM_OK;
  DeviceGuard g(k->dev);
  cudaDeviceSynchronize();
  harvest_pass_timing(k);
  if (k->graphs.pk_exec != nullptr) cudaGraphExecDestroy(k->graphs.pk_exec);
  if (k->graphs.lin_exec != nullptr) cudaGraphExecDestroy(k->graphs.lin_exec);
  if (k->graphs.loop_exec != nullptr) cudaGraphExecDestroy(k->graphs.loop_exec);
  release_batch_graph(k);
  for (auto& e : k->timing.pool) {
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  free_ws(k);
  delete k;
  return BEM_OK;
}

bem_status bem_check_guards(bem_kernel k, int64_t* bad_bytes, void* cuda_stream) {
  if (k == nullptr || bad_bytes == nullptr) {
    set_error("NULL kernel or output");
    return BEM_EINVAL;
  }
  DeviceGuard dg(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Workspace& w = k->ws;
  BEM_CUDA_TRY(cudaMemsetAsync(w.guard_bad, 0, sizeof(unsigned long long), s));
  for (int i = 0; i < w.n_guards; ++i) {
    const GuardRec& g = w.guards[i];
    k_guard_scan<<<1, (unsigned)kGuard, 0, s>>>(g.base, g.base + kGuard + g.bytes, w.guard_bad);
  }
  note_launches(w.n_guards);
  BEM_CUDA_TRY(cudaGetLastError());
  unsigned long long bad = 0;
  BEM_CUDA_TRY(cudaMemcpyAsync(&bad, w.guard_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  *bad_bytes = (int64_t)bad;
  return BEM_OK;
}

bem_status bem_debug_poke_guard(bem_kernel k, int32_t i) {
  if (k == nullptr || i < 0 || i >= k->ws.n_guards) {
    set_error("no such guarded array");
    return BEM_EINVAL;
  }
  DeviceGuard dg(k->dev);
  const GuardRec& g = k->ws.guards[i];
  BEM_CUDA_TRY(cudaMemset(g.base + kGuard + g.bytes, 0, 1));
  return BEM_OK;
}

bem_status bem_kernel_table(bem_kernel k, void* out, void* cuda_stream) {
  if (k == nullptr || out == nullptr) { set_error("NULL argument"); return BEM_EINVAL; }
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)(k->N + 1) * (k->N + 1) * sizeof(double);
  BEM_CUDA_TRY(cudaMemcpyAsync(out, k->ws.table64, bytes, cudaMemcpyDefault, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return BEM_OK;
}

bem_status bem_matvec(bem_kernel k, const void* p, void* u, void* cuda_stream) {
  Range range("bem_matvec");
  if (k == nullptr || p == nullptr || u == nullptr) { set_error("NULL argument"); return BEM_EINVAL; }
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)k->N * k->N * k->elem;
  Arg ap;
  bem_status st = stage_in(k, p, k->ws.stage_in, bytes, s, &ap);
  if (st != BEM_OK) return st;
  if (((uintptr_t)ap.dev & 15) != 0) { set_error("p must be 16-byte aligned"); return BEM_EINVAL; }
  const bool u_host = !is_device_ptr(u);
  void* ud = u_host ? k->ws.stage_out : u;
  if (((uintptr_t)ud & 15) != 0) { set_error("u must be 16-byte aligned"); return BEM_EINVAL; }
  if (k->prec == BEM_FP64)
    launch_matvec<double>(k, (const double*)ap.dev, (double*)ud, s, nullptr);
  else
    launch_matvec<float>(k, (const float*)ap.dev, (float*)ud, s, nullptr);
  BEM_CUDA_TRY(cudaGetLastError());
  if (u_host) {
    BEM_CUDA_TRY(cudaMemcpyAsync(u, ud, bytes, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
  } else if (ap.host) {
    BEM_CUDA_TRY(cudaStreamSynchronize(s));   // the host input must outlive the copy
  }
  return BEM_OK;
}

bem_status bem_solve_contact(bem_kernel k, const bem_problem* prob, void* p_out, bem_result* res,
                             void* cuda_stream) {
  Range range("bem_solve_contact");
  if (k == nullptr || res == nullptr) {
    set_error("NULL argument");
    return BEM_EINVAL;
  }
  bem_status pst = check_problem(prob);
  if (pst != BEM_OK) return pst;
  DeviceGuard g(k->dev);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const size_t n = (size_t)k->N * k->N;
  const size_t bytes = n * k->elem;
  char* vec = (char*)k->ws.vec;
  // the height map goes straight into the solver's f slot; the warm start into x
  void* fslot = vec + 5 * bytes;
  void* xslot = vec + 6 * bytes;
  const bool f_dev = is_device_ptr(prob->height);
  BEM_CUDA_TRY(cudaMemcpyAsync(fslot, prob->height, bytes, f_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  const void* pinit = nullptr;
  if (prob->p_init != nullptr) {
    const bool d = is_device_ptr(prob->p_init);
    BEM_CUDA_TRY(cudaMemcpyAsync(xslot, prob->p_init, bytes, d ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    pinit = xslot;
  }
  uint8_t* mask = k->ws.mask;
  bool mask_dev = false;
  if (prob->dgamma > 0.0) {
    if (prob->contact_mask != nullptr) {
      mask_dev = is_device_ptr(prob->contact_mask);
      BEM_CUDA_TRY(cudaMemcpyAsync(mask, prob->contact_mask, n,
                                   mask_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    } else {
      BEM_CUDA_TRY(cudaMemsetAsync(mask, 0, n, s));
    }
  }
  const bool out_host = (p_out != nullptr) && !is_device_ptr(p_out);
  void* pout_dev = out_host ? k->ws.stage_out : p_out;
  bem_status st = solve_contact_device(k, prob, fslot, pinit, mask, pout_dev, res, s);
  if (st == BEM_ECUDA || st == BEM_ENOMEM || st == BEM_EINVAL) return st;
  if (out_host) BEM_CUDA_TRY(cudaMemcpyAsync(p_out, pout_dev, bytes, cudaMemcpyDeviceToHost, s));
  if (prob->dgamma > 0.0 && prob->contact_mask != nullptr)
    BEM_CUDA_TRY(cudaMemcpyAsync(prob->contact_mask, mask, n, mask_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  BEM_CUDA_TRY(cudaStreamSynchronize(s));
  return st;
}

bem_status bem_solve_batch(int32_t n, const bem_kernel* kernels, const bem_problem* probs, void* const* p_out,
                           bem_result* res, void* cuda_stream) {
  Range range("bem_solve_batch");
  if (n < 0 || (n > 0 && (kernels == nullptr || probs == nullptr || res == nullptr))) {
    set_error("invalid batch arguments");
    return BEM_EINVAL;
  }
  if (n == 0) return BEM_OK;
  for (int32_t i = 0; i < n; ++i) {
    if (kernels[i] == nullptr) { set_error("NULL kernel in batch"); return BEM_EINVAL; }
    bem_status pst = check_problem(&probs[i]);
    if (pst != BEM_OK) return pst;
    if (kernels[i]->dev != kernels[0]->dev) { set_error("batch kernels must live on one device"); return BEM_EINVAL; }
    for (int32_t j = 0; j < i; ++j)
      if (kernels[j] == kernels[i]) { set_error("a kernel handle appears twice in the batch"); return BEM_EINVAL; }
  }
  DeviceGuard g(kernels[0]->dev);
  cudaStream_t caller = (cudaStream_t)cuda_stream;
  cudaEvent_t ready;
  BEM_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
  BEM_CUDA_TRY(cudaEventRecord(ready, caller));
  bem_status first = BEM_OK;
  // non-adhesive instances run concurrently, one precision group at a time
  for (int prec : {BEM_FP32, BEM_FP64}) {
    std::vector<int> idx;
    for (int32_t i = 0; i < n; ++i)
      if (probs[i].dgamma == 0.0 && kernels[i]->prec == prec) idx.push_back(i);
    if (idx.empty()) continue;
    const int m = (int)idx.size();
    std::vector<bem_kernel_s*> ks(m);
    std::vector<bem_problem> ps(m);
    std::vector<bem_result> rs(m);
    std::vector<cudaStream_t> strm(m);
    std::unique_ptr<bool[]> has_pinit(new bool[m]);
    for (int a = 0; a < m; ++a) {
      const int i = idx[a];
      bem_kernel_s* k = kernels[i];
      ks[a] = k;
      ps[a] = probs[i];
      strm[a] = batch_stream(k->dev, a);
      if (a < kBatchStreams) BEM_CUDA_TRY(cudaStreamWaitEvent(strm[a], ready, 0));
      const size_t bytes = (size_t)k->N * k->N * k->elem;
      char* vec = (char*)k->ws.vec;
      BEM_CUDA_TRY(cudaMemcpyAsync(vec + 5 * bytes, probs[i].height, bytes, cudaMemcpyDefault, strm[a]));
      has_pinit[a] = probs[i].p_init != nullptr;
      if (has_pinit[a])
        BEM_CUDA_TRY(cudaMemcpyAsync(vec + 6 * bytes, probs[i].p_init, bytes, cudaMemcpyDefault, strm[a]));
    }
    bem_status st = solve_batch_device(m, ks.data(), ps.data(), has_pinit.get(), rs.data(), strm.data());
    if (st != BEM_OK) {
      cudaEventDestroy(ready);
      return st;
    }
    for (int a = 0; a < m; ++a) {
      const int i = idx[a];
      res[i] = rs[a];
      if (p_out != nullptr && p_out[i] != nullptr) {
        bem_kernel_s* k = ks[a];
        const size_t bytes = (size_t)k->N * k->N * k->elem;
        BEM_CUDA_TRY(cudaMemcpyAsync(p_out[i], k->ws.vec, bytes, cudaMemcpyDefault, strm[a]));
      }
      if (rs[a].status != BEM_OK && first == BEM_OK) first = (bem_status)rs[a].status;
    }
    for (int a = 0; a < m && a < kBatchStreams; ++a) BEM_CUDA_TRY(cudaStreamSynchronize(strm[a]));
  }
  cudaEventDestroy(ready);
  // adhesive steps carry host-side outer iterations: one after another on the caller's stream
  for (int32_t i = 0; i < n; ++i) {
    if (probs[i].dgamma == 0.0) continue;
    bem_status st = bem_solve_contact(kernels[i], &probs[i], p_out ? p_out[i] : nullptr, &res[i], cuda_stream);
    if (st != BEM_OK) {
      res[i].status = st;
      if (first == BEM_OK) first = st;
    }
  }
  if (first == BEM_ENOCONV) set_error("an instance reached its iteration limit");
  if (first == BEM_ENAN) set_error("an instance met a non-finite value");
  return first;
}

}  // extern "C"
