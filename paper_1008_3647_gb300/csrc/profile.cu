// Per-kernel device timing of instrumented runs: CUDA-event pairs around each launch, with the
// launch's algorithmic bytes, aggregated by kernel class on request (ufg_profile_*).
#include <algorithm>
#include <cmath>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "line_ops.cuh"
#include "ufg_internal.h"

namespace ufg {

namespace {
struct Rec {
  std::string name;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  LaunchWork work;
  int* flags = nullptr;  // pinned snapshot of the solver flags (work.site_bytes.size() ints)
};
// Process-lifetime state (never destroyed): graph owners release their records from their own
// static destructors at exit, in an order relative to this file that C++ leaves open.
std::atomic<int> g_on{0};
std::mutex& g_mu = *new std::mutex;
std::vector<Rec>& g_recs = *new std::vector<Rec>;

// Pinned host ints handed out in order and never reused (captured graphs may still point into
// them).  Chunks are allocated only outside stream capture (a pinned allocation would invalidate
// a thread-local capture): enabling the profiler reserves one, and a launch captured after the
// current chunk has run out goes without its running-problem snapshot.
struct PinnedPool {
  std::vector<int*> chunks;
  size_t used = 0;  // ints used in the last chunk
  static constexpr size_t CHUNK = 1 << 20;
  bool grow() {
    int* p = nullptr;
    if (cudaMallocHost(&p, CHUNK * sizeof(int)) != cudaSuccess) return false;
    chunks.push_back(p);
    used = 0;
    return true;
  }
  int* take(size_t n, bool may_alloc) {
    if (n > CHUNK) return nullptr;
    if (chunks.empty() || used + n > CHUNK) {
      if (!may_alloc || !grow()) return nullptr;
    }
    int* r = chunks.back() + used;
    used += n;
    return r;
  }
  void reserve() {  // at least half a chunk free
    if (chunks.empty() || used > CHUNK / 2) grow();
  }
};
PinnedPool& g_pool = *new PinnedPool;

// Direct-launch records (their flag snapshots stay in the pool: captured graphs may still
// point into it).
void drop_records() {
  for (Rec& r : g_recs) {
    if (r.e0) cudaEventDestroy(r.e0);
    if (r.e1) cudaEventDestroy(r.e1);
  }
  g_recs.clear();
}

double resolve_bytes(const Rec& r) {
  const LaunchWork& w = r.work;
  double b = w.fixed_bytes;
  for (size_t i = 0; i < w.site_bytes.size(); ++i) {
    const bool runs = w.flag_dev == nullptr || w.exec_if < 0 || r.flags == nullptr ||
                      r.flags[i] == w.exec_if;
    if (runs) b += w.site_bytes[i];
  }
  return b;
}
}  // namespace

bool profiling() { return g_on.load(std::memory_order_relaxed) != 0; }

namespace {
// Records made while a stream is being captured become event-record (and flag-copy) nodes of
// that graph; they are re-timed after each replay of it.
std::vector<Rec>& g_pending = *new std::vector<Rec>;
std::map<cudaGraphExec_t, std::vector<Rec>>& g_graph_recs =
    *new std::map<cudaGraphExec_t, std::vector<Rec>>;
struct Agg {
  long long launches = 0;
  double ms = 0.0, bytes = 0.0;
};
std::map<std::string, Agg>& g_agg = *new std::map<std::string, Agg>;  // harvested replays

void destroy(std::vector<Rec>& v) {
  for (Rec& r : v) {
    if (r.e0) cudaEventDestroy(r.e0);
    if (r.e1) cudaEventDestroy(r.e1);
  }
  v.clear();
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive;
}
}  // namespace

KTimer::KTimer(const std::string& name, cudaStream_t st, LaunchWork work) : st_(st) {
  if (!profiling()) return;
  Rec r;
  r.name = name;
  r.work = std::move(work);
  const bool cap = capturing(st);
  std::lock_guard<std::mutex> lk(g_mu);
  if (r.work.flag_dev != nullptr && r.work.exec_if >= 0 && !r.work.site_bytes.empty()) {
    r.flags = g_pool.take(r.work.site_bytes.size(), !cap);
    if (r.flags != nullptr &&
        cudaMemcpy2DAsync(r.flags, sizeof(int), r.work.flag_dev, r.work.stride, sizeof(int),
                          r.work.site_bytes.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      r.flags = nullptr;
  }
  if (cudaEventCreate(&r.e0) != cudaSuccess || cudaEventCreate(&r.e1) != cudaSuccess) {
    if (r.e0) cudaEventDestroy(r.e0);
    return;  // timing is best effort: the launch itself proceeds
  }
  cap_ = cap;
  if (cap) {
    cudaEventRecordWithFlags(r.e0, st, cudaEventRecordExternal);
    idx_ = (long long)g_pending.size();
    g_pending.push_back(std::move(r));
  } else {
    cudaEventRecord(r.e0, st);
    idx_ = (long long)g_recs.size();
    g_recs.push_back(std::move(r));
  }
}

KTimer::~KTimer() {
  if (idx_ < 0) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap_) {
    if (idx_ < (long long)g_pending.size())
      cudaEventRecordWithFlags(g_pending[(size_t)idx_].e1, st_, cudaEventRecordExternal);
  } else if (idx_ < (long long)g_recs.size()) {
    cudaEventRecord(g_recs[(size_t)idx_].e1, st_);
  }
}

void profile_capture_begin() {
  std::lock_guard<std::mutex> lk(g_mu);
  destroy(g_pending);
}

void profile_capture_end(cudaGraphExec_t ex) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (ex == nullptr || g_pending.empty()) {
    destroy(g_pending);
    return;
  }
  destroy(g_graph_recs[ex]);
  g_graph_recs[ex] = std::move(g_pending);
  g_pending.clear();
}

void profile_after_replay(cudaGraphExec_t ex, cudaStream_t st) {
  if (!profiling()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_graph_recs.find(ex);
  if (it == g_graph_recs.end() || cudaStreamSynchronize(st) != cudaSuccess) return;
  for (const Rec& r : it->second) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) continue;
    Agg& a = g_agg[r.name];
    a.launches += 1;
    a.ms += ms;
    a.bytes += resolve_bytes(r);
  }
}

void profile_graph_destroyed(cudaGraphExec_t ex) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_graph_recs.find(ex);
  if (it == g_graph_recs.end()) return;
  destroy(it->second);
  g_graph_recs.erase(it);
}

std::string slice_kernel_name(const SliceCall& c, int N) {
  static const char* fam[] = {"kin", "fwd", "inv", "m1w", "Q"};
  std::string s = "slice ";
  s += (c.fam >= 0 && c.fam <= 4) ? fam[c.fam] : "?";
  if (c.fam == FAM_Q) {
    if (c.U || c.V) s += "+uv";
    if (c.want_dotP || c.want_self) s += "+dot";
  } else if (c.fam != FAM_M1W) {
    if (c.pre) s += "+pre";
    if (c.bkpre) s += "+bkpre";
    if (c.bkpost) s += "+bkpost";
    if (c.id) s += "+id";
    if (c.post) s += "+post";
    if (c.post2) s += "+post2";
    if (c.U || c.V) s += "+uv";
    if (c.want_dotP || c.want_self) s += "+dot";
    if (c.prep_out) s += "+prep";
  } else {
    s += c.shift > 0 ? "T" : "";
    if (c.m1w_full) s += (c.want_dotP || c.want_self) ? "+full+dot" : "+full";
  }
  s += " N" + std::to_string(N) + (c.prec ? " f32" : (c.emulate64 ? " f64 as double-float" : " f64"));
  return s;
}

double slice_bytes_per_site(const SliceCall& c) {
  const double es = c.prec ? 4.0 : 8.0;
  int site_arrays = 2;  // input and output
  if (c.pre) ++site_arrays;
  if (c.id) ++site_arrays;
  if (c.post) ++site_arrays;
  if (c.post2) ++site_arrays;
  if (c.U) ++site_arrays;
  if (c.V) ++site_arrays;
  if (c.want_dotP && c.dotP) ++site_arrays;
  if (c.prep_out) site_arrays += 3;  // r and v read, p written
  return es * site_arrays;
}

double slice_bytes_per_problem(const SliceCall& c, int N) {
  const int mode_tables = (c.bkpre ? 1 : 0) + (c.bkpost ? 1 : 0);
  return (c.prec ? 4.0 : 8.0) * mode_tables * std::pow((double)N, c.dim);
}

}  // namespace ufg

using namespace ufg;

extern "C" ufg_status ufg_profile_enable(int on) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_mu);
  if (on) {
    cudaDeviceSynchronize();
    drop_records();
    g_agg.clear();
    g_pool.reserve();
  }
  g_on.store(on ? 1 : 0);
  return UFG_OK;
}

extern "C" ufg_status ufg_profile_read(ufg_kernel_stat* out, int max, int* n) {
  clear_error();
  if (n == nullptr || max < 0 || (max > 0 && out == nullptr)) {
    set_error("profile_read: need n, and out when max > 0");
    return UFG_INVALID_ARG;
  }
  UFG_CUDA(cudaDeviceSynchronize());
  std::map<std::string, Agg> agg;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    agg = g_agg;
    for (const Rec& r : g_recs) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) continue;
      Agg& a = agg[r.name];
      a.launches += 1;
      a.ms += ms;
      a.bytes += resolve_bytes(r);
    }
  }
  std::vector<std::pair<std::string, Agg>> v(agg.begin(), agg.end());
  std::sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.second.ms > y.second.ms; });
  *n = (int)v.size();
  for (int i = 0; i < max && i < (int)v.size(); ++i) {
    std::memset(&out[i], 0, sizeof(ufg_kernel_stat));
    std::strncpy(out[i].name, v[(size_t)i].first.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = v[(size_t)i].second.launches;
    out[i].total_ms = v[(size_t)i].second.ms;
    out[i].bytes = v[(size_t)i].second.bytes;
  }
  return UFG_OK;
}

// ---- arithmetic peak of this GPU (roofline denominators of the FP64 and FP32 applies) --------
namespace ufg {
namespace {

// Each thread runs 8 independent multiply-add chains for `iters` rounds; the chains start from
// values only the caller knows, and their sum is stored, so nothing can be folded away.
template <typename R>
__global__ void __launch_bounds__(256) fma_rate_kernel(R seed, int iters, R* out) {
  R a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = seed + R(threadIdx.x * 8 + k) * R(1e-7);
  const R m = R(0.999999), c = R(1e-9);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fmadd(a[k], m, c);
  }
  R s = R(0);
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
ufg_status fma_rate(cudaStream_t st, double* tflops) {
  int dev = 0, sms = 0, per_sm = 0;
  UFG_CUDA(cudaGetDevice(&dev));
  UFG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  UFG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_rate_kernel<R>, 256, 0));
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const int iters = sizeof(R) == 8 ? 4096 : 65536;
  R* out = nullptr;
  UFG_TRY(dev_alloc(&out, (size_t)blocks * 256));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  fma_rate_kernel<R><<<blocks, 256, 0, st>>>(R(1), iters, out);  // warm-up
  cudaEventRecord(e0, st);
  const int reps = 5;
  for (int r = 0; r < reps; ++r) fma_rate_kernel<R><<<blocks, 256, 0, st>>>(R(1), iters, out);
  cudaEventRecord(e1, st);
  note_launches(reps + 1);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(out);
  if (e != cudaSuccess) return cuda_fail(e, "FMA-rate kernel");
  const double flops = 2.0 * 8.0 * iters * 256.0 * blocks * reps;
  *tflops = flops / (ms * 1e-3) / 1e12;
  return UFG_OK;
}

}  // namespace
}  // namespace ufg

extern "C" ufg_status ufg_measure_fma_rate(int precision, void* stream, double* tflops) {
  clear_error();
  if (tflops == nullptr || (precision != UFG_FP64 && precision != UFG_FP32)) {
    set_error("measure_fma_rate: need tflops and precision UFG_FP64 or UFG_FP32");
    return UFG_INVALID_ARG;
  }
  return precision == UFG_FP64 ? fma_rate<double>(as_stream(stream), tflops)
                               : fma_rate<float>(as_stream(stream), tflops);
}
