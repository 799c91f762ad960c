// Host driver of PHSVDS on one GB300 and the C ABI (include/phsvds.h).
//
// Stage 1 (Algorithm 1): block GD+k on C = A^T A.  Stage 2 (Algorithm 2): GD
// outer loop on B = [0 A^T; A 0] with the refined projection through an
// incrementally updated QR of W - s V.  Every arithmetic step runs in the
// kernels of k_sparse.cu / k_tall.cu / k_small.cu; the host only sequences
// launches and reads back the few scalars that decide locking and restarts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "phsvds.h"

namespace ph {

constexpr int LD = 64;                    // leading dimension of the small matrices
constexpr double EPS64 = 2.220446049250313e-16;
constexpr double EPS32 = 1.1920928955078125e-07;
constexpr uint64_t RS_INIT = 0x1000, RS_BREAK = 0x2000, RS_U = 0x3000, RS_NORM = 0x4000;
constexpr double JAC_TOL = 5e-17;         // Jacobi threshold for pairs touching a target, relative to ||H||
constexpr double TOL_MARGIN = 0.9;        // stopping tests use 0.9 delta: the residual the test sees and an
                                          // independent recomputation differ by rounding of order eps ||C||
constexpr double JAC_REL = 1e-8;          // relative threshold of the other pairs (they span the restart space)
constexpr int W_REFRESH = 16;             // stage-1 restarts between recomputations of W = C V
constexpr double EIG32_GATE = 1e-5;       // FP32-first projected solve when the targets are >= this x theta_max
constexpr double JAC_REL32 = 1e-6;        // its FP64 clean-up: relative threshold of the non-target pairs
constexpr int RI_MAXIT = 24;               // stage 2: inverse-iteration steps for the refined vector (at most)
constexpr double RI_TAU = 1e-10;          // ... which stop once ||R x|| falls by less than this (relative)
constexpr double STAG_NEAR = 2.0;         // stage-1 stagnation: residual within 2x of its tolerance ...
constexpr double STAG_RATIO = 100.0;      // ... or within 100x for STAG_LONG iterations without halving
constexpr int64_t STAG_LONG = 2000;

struct PhError {
  phsvds_status st;
  std::string msg;
};

#define CUCHK(x)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) throw PhError{e_ == cudaErrorMemoryAllocation ? PHSVDS_ERR_OOM : PHSVDS_ERR_CUDA, \
                                         std::string(#x) + ": " + cudaGetErrorString(e_)};      \
  } while (0)

// Device allocation owned by a solve (stream-ordered, from the handle's
// memory pool, which keeps its memory between solves).
struct Pool {
  cudaStream_t s;
  cudaMemPool_t mp;
  std::vector<void*> ptrs;
  Pool(cudaStream_t st, cudaMemPool_t m) : s(st), mp(m) {}
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    if (count == 0) count = 1;
    if (mp)
      CUCHK(cudaMallocFromPoolAsync(&p, sizeof(T) * count, mp, s));
    else
      CUCHK(cudaMallocAsync(&p, sizeof(T) * count, s));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Pool() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// An SpMM schedule picked by the autotuner for one matrix shape and block
// width (kept by the handle, reused by its later solves of that shape).
struct SpmmPlan {
  int64_t m = 0, n = 0, nnz = 0;
  int b = 0, bytes = 0, deterministic = 0;
  int schedule = 2, lanes = 0, lanes_a = 0, lanes_at = 0;
};

// The fixed-order reduction scratch of one solve (3 MiB from its pool) made
// this host thread's for the scope's life; the previous scratch comes back
// at the end (a solve inside Algorithm 3's driver).  A solve's reductions
// are serial on its stream, so one scratch serves them all.
constexpr size_t RED_WS_DOUBLES = 393216;
struct RedScope {
  RedWs prev;
  size_t prev_cap;
  RedScope(Pool& pool, cudaStream_t s);
  ~RedScope();
};

}  // namespace ph

struct phsvds_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  unsigned char* host = nullptr;  // pinned readback / upload area
  size_t host_bytes = 0;
  std::vector<ph::SpmmPlan> plans;  // autotuned SpMM schedules of earlier solves
  // device memory of the solves: a pool that keeps what it has mapped until
  // the handle is destroyed, so that repeated solves do not map and unmap
  // their workspaces (the default pool returns memory at every synchronise)
  cudaMemPool_t mempool = nullptr;
};

namespace ph {

int handle_device(const phsvds_ctx* h) { return h->device; }
cudaStream_t handle_stream(const phsvds_ctx* h) { return h->stream; }

// Pinned staging area of the context (readbacks of a few scalars per iteration).
struct Host {
  phsvds_ctx* c;
  unsigned char* base;
  size_t bytes;
  explicit Host(phsvds_ctx* cc) : c(cc), base(cc->host), bytes(cc->host_bytes) {}
  template <typename T> T* at(size_t off_bytes) { return reinterpret_cast<T*>(base + off_bytes); }
};

// ---- instrumentation (per host thread)
static thread_local int64_t g_launch_count = 0;
void count_launch() { ++g_launch_count; }
static thread_local double g_work[2][PROF_NALL] = {};  // [0] flops, [1] bytes per kernel class
// scratch of the fixed-order cross-block reductions of this host thread's solve
static thread_local RedWs g_red{};
static thread_local size_t g_red_cap = 0;
RedWs red_ws(size_t doubles) { return doubles <= g_red_cap ? g_red : RedWs{}; }
void set_red_ws(double* ws, size_t cap) {
  g_red = RedWs{ws};
  g_red_cap = ws ? cap : 0;
}
void count_work(int cat, double flops, double bytes) {
  g_work[0][cat] += flops;
  g_work[1][cat] += bytes;
}

struct Profiler {
  bool on = false;
  int depth[PROF_NALL] = {};
  std::vector<cudaEvent_t> ev;
  std::vector<int> evcat;
  size_t used = 0;
  double acc_ms[PROF_NALL] = {};  // intervals already folded in (the buffer is reused)
  int64_t acc_n[PROF_NALL] = {};
  void start(size_t cap) {
    on = true;
    for (int c = 0; c < PROF_NALL; ++c) depth[c] = 0, acc_ms[c] = 0.0, acc_n[c] = 0;
    while (ev.size() < cap) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      ev.push_back(e);
    }
    evcat.assign(ev.size(), 0);
    used = 0;
  }
  // times of the recorded intervals into acc (waits for the last one)
  void fold() {
    for (size_t i = 0; i + 1 < used; i += 2) {
      float t = 0.f;
      if (cudaEventSynchronize(ev[i + 1]) == cudaSuccess && cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess) {
        acc_ms[evcat[i]] += t;
        acc_n[evcat[i]] += 1;
      }
    }
    used = 0;
  }
  void mark(cudaStream_t s, int cat, bool begin) {
    if (!on) return;
    if (begin && depth[cat]++ > 0) return;
    if (!begin && --depth[cat] > 0) return;
    if (!begin && (used & 1) == 0) return;  // unmatched end
    if (begin && (used & 1) == 1) return;   // another class is open: skip nested
    if (begin && used + 2 > ev.size()) fold();  // full: fold the finished intervals, reuse the events
    if (used >= ev.size()) return;
    cudaEventRecord(ev[used], s);
    evcat[used] = cat;
    ++used;
  }
  void finish(double* ms, int64_t* cnt) {
    fold();
    on = false;
    for (int c = 0; c < PROF_NALL; ++c) ms[c] += acc_ms[c], cnt[c] += acc_n[c];
  }
};
static thread_local Profiler g_prof;
void prof_begin(cudaStream_t s, int cat) { g_prof.mark(s, cat, true); }
void prof_end(cudaStream_t s, int cat) { g_prof.mark(s, cat, false); }

static bool trace_on() {
  static const bool t = getenv("PHSVDS_TRACE") != nullptr;  // initialised once, thread-safe
  return t;
}

static void sync(cudaStream_t s) {
  CUCHK(cudaGetLastError());
  CUCHK(cudaStreamSynchronize(s));
}

template <typename T> static void zero(cudaStream_t s, T* p, size_t count) {
  if (count) CUCHK(cudaMemsetAsync(p, 0, sizeof(T) * count, s));
}

RedScope::RedScope(Pool& pool, cudaStream_t s) : prev(g_red), prev_cap(g_red_cap) {
  (void)s;
  set_red_ws(pool.get<double>(RED_WS_DOUBLES), RED_WS_DOUBLES);
}
RedScope::~RedScope() {
  g_red = prev;
  g_red_cap = prev_cap;
}

// ---------------------------------------------------------------------------
// The matrix on the device
// ---------------------------------------------------------------------------
struct DevA {
  int m = 0, n = 0;
  int64_t nnz = 0;
  int *rp = nullptr, *ci = nullptr, *cp = nullptr, *ri = nullptr;
  double *va = nullptr, *cv = nullptr, *diagC = nullptr;
  float *va32 = nullptr, *cv32 = nullptr;
  SparseView<double> A64, At64;
  SparseView<float> A32, At32;
  double *Z64 = nullptr;
  float *Z32 = nullptr;
};

static void upload_matrix(phsvds_ctx* ctx, Pool& pool, DevA& d, int64_t m, int64_t n, int64_t nnz, const int64_t* rp,
                          const int32_t* ci, const double* va, int on_dev, bool need32, bool need_diag, int bmax) {
  cudaStream_t s = ctx->stream;
  d.m = (int)m;
  d.n = (int)n;
  d.nnz = nnz;
  int64_t* rp64 = pool.get<int64_t>(m + 1);
  d.rp = pool.get<int>(m + 1);
  d.ci = pool.get<int>(nnz);
  d.va = pool.get<double>(nnz);
  const cudaMemcpyKind kind = on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUCHK(cudaMemcpyAsync(rp64, rp, sizeof(int64_t) * (m + 1), kind, s));
  if (nnz) {
    CUCHK(cudaMemcpyAsync(d.ci, ci, sizeof(int) * nnz, kind, s));
    CUCHK(cudaMemcpyAsync(d.va, va, sizeof(double) * nnz, kind, s));
  }
  int* flags = pool.get<int>(2);
  zero(s, flags, 2);
  rowptr_check(s, d.m, nnz, rp64, d.rp, flags);
  validate_rows(s, d.m, d.n, d.rp, d.ci, d.va, flags);
  Host h(ctx);
  CUCHK(cudaMemcpyAsync(h.at<int>(0), flags, sizeof(int), cudaMemcpyDeviceToHost, s));
  sync(s);
  const int f = *h.at<int>(0);
  if (f & 1) throw PhError{PHSVDS_ERR_INVALID, "invalid CSR structure (row_ptr or column indices)"};
  if (f & 2) throw PhError{PHSVDS_ERR_NAN, "A holds a NaN or Inf value"};
  d.cp = pool.get<int>(n + 1);
  d.ri = pool.get<int>(nnz);
  d.cv = pool.get<double>(nnz);
  int* work = pool.get<int>(n);
  csr_to_csc<double>(s, d.m, d.n, nnz, d.rp, d.ci, d.va, d.cp, d.ri, d.cv, work);
  d.A64 = SparseView<double>{d.m, d.n, nnz, d.rp, d.ci, d.va};
  d.At64 = SparseView<double>{d.n, d.m, nnz, d.cp, d.ri, d.cv};
  d.Z64 = pool.get<double>((size_t)m * bmax);
  if (need32) {
    d.va32 = pool.get<float>(nnz);
    d.cv32 = pool.get<float>(nnz);
    to_float(s, nnz, d.va, d.va32);
    to_float(s, nnz, d.cv, d.cv32);
    d.A32 = SparseView<float>{d.m, d.n, nnz, d.rp, d.ci, d.va32};
    d.At32 = SparseView<float>{d.n, d.m, nnz, d.cp, d.ri, d.cv32};
    d.Z32 = pool.get<float>((size_t)m * bmax);
  }
  if (need_diag) {
    d.diagC = pool.get<double>(n);
    col_norms2(s, d.n, d.cp, d.cv, d.diagC);
  }
}

// C X = A^T (A X) on a row-major block of b in {1,2,4,8} vectors.
template <typename T> struct COp {
  const SparseView<T>* A;
  const SparseView<T>* At;
  T* Z;
  int n;
  int schedule;      // 1 fused atomic, 2 two-phase
  int lanes = 0;     // fused: lanes per row of A (0 = from the mean row length)
  int lanes_a = 0;   // two-phase: lanes per row of A (Z = A X) and of A^T (Y = A^T Z)
  int lanes_at = 0;
  mutable int64_t calls = 0;
  void apply(cudaStream_t s, int b, const T* X, T* Y) const {
    ++calls;
    if (schedule == 1)
      ata_fused<T>(s, *A, n, b, X, Y, lanes);
    else
      ata_two_phase<T>(s, *A, *At, b, X, Y, Z, lanes_a, lanes_at);
  }
};

// B X = [A^T X_u; A X_v] on a row-major block of b vectors of length n + m
// (the [v; u] order of the augmented vectors), as GD+k on B needs it
// (Algorithm 3).
struct BOp {
  const SparseView<double>* A;
  const SparseView<double>* At;
  int m, n;
  void apply(cudaStream_t s, int b, const double* X, double* Y) const {
    csr_spmm<double>(s, *At, b, X + (size_t)n * b, Y);
    csr_spmm<double>(s, *A, b, X, Y + (size_t)n * b);
  }
};

// Mean time (ms) of f() over 3 launches after one warm-up, on stream s.
template <typename F>
static float time_launches(cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, F&& f) {
  f();
  CUCHK(cudaEventRecord(e0, s));
  for (int r = 0; r < 3; ++r) f();
  CUCHK(cudaEventRecord(e1, s));
  CUCHK(cudaEventSynchronize(e1));
  float ms = 0;
  CUCHK(cudaEventElapsedTime(&ms, e0, e1));
  return ms / 3;
}

// Candidate group widths around the one picked from the mean row length;
// for 32-byte rows also each width with the row gathers kept out of L1
// (negative value).
static std::vector<int> lane_candidates(double avg, bool rows32) {
  const int l0 = lanes_for(avg);
  std::vector<int> c;
  for (int l : {l0 / 2, l0, l0 * 2})
    if (l >= 1 && l <= 16 && std::find(c.begin(), c.end(), l) == c.end()) c.push_back(l);
  if (rows32)
    for (size_t i = 0, k = c.size(); i < k; ++i) c.push_back(-c[i]);
  return c;
}

// The SpMM autotuner: times the fused schedule over its lane widths, each
// phase of the two-phase schedule over its lane widths, then the best
// two-phase pair, on this matrix and block width, and keeps the fastest.
template <typename T>
static COp<T> autotune_spmm(cudaStream_t s, Pool& pool, const SparseView<T>& A, const SparseView<T>& At, T* Z, int n,
                            int b, bool deterministic) {
  T* X = pool.get<T>((size_t)n * b);
  T* Y = pool.get<T>((size_t)n * b);
  fill_random<T>(s, n * b, X, 7, 0x77);
  cudaEvent_t e0, e1;
  CUCHK(cudaEventCreate(&e0));
  CUCHK(cudaEventCreate(&e1));
  COp<T> best{&A, &At, Z, n, 2};
  float tbest = 1e30f;
  const bool rows32 = sizeof(T) * b == 32;
  // the fused schedule sums with atomics (order not fixed): only when results
  // need not repeat bit for bit
  if (!deterministic)
    for (int l : lane_candidates(A.avg_row(), rows32)) {
      COp<T> op{&A, &At, Z, n, 1, l};
      const float t = time_launches(s, e0, e1, [&] { op.apply(s, b, X, Y); });
      if (t < tbest) tbest = t, best = op;
    }
  int la = 0, lat = 0;
  float ta = 1e30f, tat = 1e30f;
  for (int l : lane_candidates(A.avg_row(), rows32)) {
    const float t = time_launches(s, e0, e1, [&] { csr_spmm<T>(s, A, b, X, Z, l); });
    if (t < ta) ta = t, la = l;
  }
  for (int l : lane_candidates(At.avg_row(), rows32)) {
    const float t = time_launches(s, e0, e1, [&] { csr_spmm<T>(s, At, b, Z, Y, l); });
    if (t < tat) tat = t, lat = l;
  }
  COp<T> two{&A, &At, Z, n, 2, 0, la, lat};
  const float t2 = time_launches(s, e0, e1, [&] { two.apply(s, b, X, Y); });
  // the two-phase schedule sums in a fixed order (the fused one's atomics do
  // not): keep it unless the fused schedule is clearly faster, so repeated
  // solves take the same path
  if (t2 <= tbest / 0.85f) best = two;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best.calls = 0;
  return best;
}

static inline int spmm_width(int nb) { return nb >= 8 ? 8 : nb >= 4 ? 4 : nb >= 2 ? 2 : 1; }

// The autotuned schedule for this matrix shape and block width: the handle's
// plan from an earlier solve of the same m, n, nnz, b and precision, else a
// fresh autotune, which is then kept.  Any plan computes the same product
// (the schedules differ only in summation order), so a plan taken from
// another matrix of the same shape costs at most speed.
template <typename T>
static COp<T> tuned_spmm(phsvds_ctx* ctx, Pool& pool, const SparseView<T>& A, const SparseView<T>& At, T* Z, int n,
                         int b, bool* cached, bool deterministic) {
  for (const SpmmPlan& p : ctx->plans)
    if (p.m == A.nrows && p.n == n && p.nnz == A.nnz && p.b == b && p.bytes == (int)sizeof(T) &&
        p.deterministic == (int)deterministic) {
      *cached = true;
      return COp<T>{&A, &At, Z, n, p.schedule, p.lanes, p.lanes_a, p.lanes_at};
    }
  COp<T> op = autotune_spmm<T>(ctx->stream, pool, A, At, Z, n, b, deterministic);
  SpmmPlan p;
  p.m = A.nrows, p.n = n, p.nnz = A.nnz, p.b = b, p.bytes = (int)sizeof(T), p.deterministic = (int)deterministic;
  p.schedule = op.schedule, p.lanes = op.lanes, p.lanes_a = op.lanes_a, p.lanes_at = op.lanes_at;
  if (ctx->plans.size() >= 64) ctx->plans.erase(ctx->plans.begin());
  ctx->plans.push_back(p);
  *cached = false;
  return op;
}

// Jacobi frame of the projected problem, rebuilt from the exact projected
// matrix Ht (basis coordinates): ns_steps Newton-Schulz steps
// S <- S (3I - S^T S)/2 keep the accumulated rotation orthonormal (each step
// squares its loss of orthogonality), then Aw = S^T Ht S.  With ns_steps < 0
// the rotation is the identity and the frame is Ht itself.
static void frame_from_true(cudaStream_t s, int j, const double* Ht, double* S, double* Aw, double* w1, double* w2,
                            int ns_steps) {
  if (ns_steps < 0) {
    CUCHK(cudaMemcpy2DAsync(Aw, LD * sizeof(double), Ht, LD * sizeof(double), j * sizeof(double), j,
                            cudaMemcpyDeviceToDevice, s));
    return;
  }
  for (int it = 0; it < ns_steps; ++it) {
    small_gemm_tn(s, j, j, j, S, LD, S, LD, w1, LD);
    ns_factor(s, j, w1, LD);
    small_gemm_nn(s, j, j, j, S, LD, w1, LD, w2, LD);
    CUCHK(cudaMemcpy2DAsync(S, LD * sizeof(double), w2, LD * sizeof(double), j * sizeof(double), j,
                            cudaMemcpyDeviceToDevice, s));
  }
  small_gemm_nn(s, j, j, j, Ht, LD, S, LD, w1, LD);
  small_gemm_tn(s, j, j, j, S, LD, w1, LD, Aw, LD);
  symmetrise(s, j, Aw, LD);
}

// Mixed-precision Rayleigh-Ritz eigensolve on GB300 (one SM's FP64 pipe is
// ~60x slower than its FP32 pipe): an FP32 cyclic Jacobi pass does the large
// rotations of the warm frame, S <- S Sf is re-orthonormalised and the exact
// FP64 frame S^T Ht S rebuilt, and (when fp64_cleanup) an FP64 Jacobi pass,
// tight only on pairs touching the targets, brings the targeted Ritz pairs to
// FP64 accuracy.  theta = diagonal of the final frame, S = its rotation.
static void eig_mixed(cudaStream_t s, int j, const double* Ht, double* S, double* Aw, double* Sf, double* theta,
                      double* w1, double* w2, bool s_ident, bool fp64_cleanup, int ntarget, int tmode, double tshift,
                      int* counters, double rel = JAC_REL, bool targets_only = false) {
  frame_from_true(s, j, Ht, S, Aw, w1, w2, s_ident ? -1 : 0);
  jacobi_eig32_ld(s, j, Aw, LD, Sf, LD, theta, 1e-6, 30, counters, counters + 1);
  if (s_ident) {
    CUCHK(cudaMemcpy2DAsync(S, LD * sizeof(double), Sf, LD * sizeof(double), j * sizeof(double), j,
                            cudaMemcpyDeviceToDevice, s));
  } else {
    small_gemm_nn(s, j, j, j, S, LD, Sf, LD, w2, LD);
    CUCHK(cudaMemcpy2DAsync(S, LD * sizeof(double), w2, LD * sizeof(double), j * sizeof(double), j,
                            cudaMemcpyDeviceToDevice, s));
  }
  frame_from_true(s, j, Ht, S, Aw, w1, w2, fp64_cleanup ? 2 : 1);
  if (fp64_cleanup && targets_only)
    jacobi_eig_targets_ld(s, j, Aw, LD, S, LD, theta, JAC_TOL, 60, counters + 2, ntarget, tmode, tshift,
                          counters + 3);
  else if (fp64_cleanup)
    jacobi_eig_ld(s, j, Aw, LD, S, LD, theta, JAC_TOL, 60, counters + 2, rel, ntarget, tmode, tshift,
                  counters + 3);
  else
    jacobi_eig32_ld(s, j, Aw, LD, Sf, LD, theta, 1e-6, 0, nullptr, nullptr);  // theta = diag of the rebuilt frame
}

// Ht = V^T W recomputed from the tall basis after a transform (j x j, FP64
// accumulation): no rounding drift of the projected matrix survives a restart.
template <typename T>
static void gram_full(cudaStream_t s, int n, const T* V, T* W, int j, double* Ht, double* tmp) {
  Basis<T> P{V, n, j, nullptr, 0, 0};
  for (int c = 0; c < j; c += 8) {
    const int w = std::min(8, j - c);
    zero(s, tmp, (size_t)j * w);
    cgs_pass<T>(s, n, P, W + (size_t)c * n, n, w, nullptr, tmp, nullptr);
    CUCHK(cudaMemcpy2DAsync(Ht + (size_t)c * LD, LD * sizeof(double), tmp, j * sizeof(double), j * sizeof(double), w,
                            cudaMemcpyDeviceToDevice, s));
  }
  symmetrise(s, j, Ht, LD);
}

// ---------------------------------------------------------------------------
// Stage 1: block GD+k on C (storage precision T)
// ---------------------------------------------------------------------------
// Cached CUDA graphs of the launch-heavy, host-sync-free segments of an outer
// iteration, keyed by everything host-side the segment depends on (the
// buffers of a solve stay put).  A key's first occurrence runs eagerly (so
// function attributes and lazy module loads happen outside any capture), its
// second is captured and instantiated, later ones replay the graph.  If a
// capture cannot be made (a caller stream that cannot be captured, say) the
// cache switches itself off and every segment runs eagerly.
struct GraphCache {
  struct Entry {
    int seen = 0;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    double work[2][PROF_NALL] = {};  // algorithmic work of one replay
  };
  static void add_work(const Entry& e) {
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < PROF_NALL; ++c) g_work[a][c] += e.work[a][c];
  }
  std::unordered_map<uint64_t, Entry> map;
  bool enabled = true;
  ~GraphCache() {
    for (auto& kv : map)
      if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
  }
  template <typename F>
  void run(cudaStream_t s, uint64_t key, F&& issue) {
    if (!enabled) return issue();
    Entry& e = map[key];
    if (e.exec) {
      CUCHK(cudaGraphLaunch(e.exec, s));
      g_launch_count += e.launches;
      add_work(e);
      return;
    }
    if (e.seen++ == 0) return issue();
    const int64_t l0 = g_launch_count;
    double w0[2][PROF_NALL];
    std::memcpy(w0, g_work, sizeof(w0));
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      enabled = false;
      return issue();
    }
    try {
      issue();
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(s, &g);
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t g = nullptr;
    cudaError_t st = cudaStreamEndCapture(s, &g);
    if (st == cudaSuccess && g) st = cudaGraphInstantiate(&e.exec, g, 0);
    if (g) cudaGraphDestroy(g);
    const int64_t captured = g_launch_count - l0;
    g_launch_count = l0;
    for (int a = 0; a < 2; ++a)
      for (int c = 0; c < PROF_NALL; ++c) e.work[a][c] = g_work[a][c] - w0[a][c];
    std::memcpy(g_work, w0, sizeof(w0));
    if (st != cudaSuccess || !e.exec) {  // nothing ran: switch off and run eagerly
      cudaGetLastError();
      e.exec = nullptr;
      enabled = false;
      return issue();
    }
    e.launches = captured;
    CUCHK(cudaGraphLaunch(e.exec, s));
    g_launch_count += e.launches;
    add_work(e);
  }
};

// Jacobi-Davidson corrections of stage 1 (the JDQMR form of Sec. 4): the
// correction equation (I - QQ^T)(C - theta I)(I - QQ^T) t = r, Q = [locked
// vectors, x], of each targeted Ritz pair, solved for the block at once by
// MINRES.  In the FP64 continuation of the mixed-precision stage 1 the solve
// runs in FP32 with the FP32 products with C (InnerJD<float>); in the FP64
// method (opts.stage1_inner) in FP64 (InnerJD<double>).  The outer
// Rayleigh-Ritz, the residuals that decide convergence and the
// orthogonalisation of t into the basis are FP64 either way.
// With the Jacobi preconditioner D = diag(C) (Sec. 4's preconditioned JDQMR)
// the equation is solved in the scaled variable y = D^{1/2} t:
// D^{-1/2} P (C - theta I) P D^{-1/2} y = D^{-1/2} r, a symmetric system, with
// P = I - QQ^T and Q = [locked vectors, all q Ritz vectors of the block] on
// both sides (the scaled vectors leave the complement of Q, so the
// projection is applied to the operator's input as well); t = D^{-1/2} y.
struct InnerSolver {
  int64_t steps = 0, solves = 0;
  // Tb (n x q, FP64): residuals on entry, corrections on return.  Xu: the q
  // Ritz vectors, theta (device, q): their Ritz values, Xl: nl locked vectors;
  // dC (device, n): diag(C) for the scaled form (null: unscaled), entries
  // below guard raised to it.
  virtual void solve(phsvds_ctx* ctx, int q, double* Tb, const double* Xu, const double* theta, const double* Xl,
                     int nl, const double* dC = nullptr, double guard = 0.0) = 0;
  // the same with FP32 storage (the FP32 stage of the mixed form)
  virtual void solve(phsvds_ctx* ctx, int q, float* Tb, const float* Xu, const double* theta, const float* Xl, int nl,
                     const double* dC = nullptr, double guard = 0.0) = 0;
  virtual ~InnerSolver() = default;
};

template <typename T>
struct InnerJD : InnerSolver {
  cudaStream_t s;
  int n, maxit, chunk = 5;
  double tol;
  COp<T> op;
  T *R, *r1, *r2, *v, *sol, *w1, *w2, *X, *Cv, *Xrm, *Yrm, *Xq, *U, *ds;
  double *acc, *sc, *g1;
  GraphCache graphs;
  InnerJD(phsvds_ctx* c, Pool& pool, int n_, int kmax, COp<T> op_, int maxit_, double tol_, bool use_graphs)
      : s(c->stream), n(n_), maxit(maxit_), tol(tol_), op(op_) {
    const size_t nn = (size_t)n;
    R = pool.get<T>(nn * 8);
    r1 = pool.get<T>(nn * 8);
    r2 = pool.get<T>(nn * 8);
    v = pool.get<T>(nn * 8);
    sol = pool.get<T>(nn * 8);
    w1 = pool.get<T>(nn * 8);
    w2 = pool.get<T>(nn * 8);
    X = pool.get<T>(nn * 8);
    Cv = pool.get<T>(nn * 8);
    Xrm = pool.get<T>(nn * 8);
    Yrm = pool.get<T>(nn * 8);
    Xq = pool.get<T>(nn * (kmax + 8));
    U = pool.get<T>(nn * 8);
    ds = pool.get<T>(nn);
    acc = pool.get<double>(32 + 8 * 64);
    sc = pool.get<double>(JD_NSCALAR * 8);
    g1 = pool.get<double>(8 * 64);
    graphs.enabled = use_graphs;
  }
  // the caller's vectors into the solve's precision, and the result back
  template <typename S>
  void in(int64_t cnt, const S* src, T* dst) {
    if constexpr (sizeof(S) == sizeof(T))
      CUCHK(cudaMemcpyAsync(dst, src, sizeof(T) * cnt, cudaMemcpyDeviceToDevice, s));
    else if constexpr (sizeof(T) == 4)
      convert_f64_to_f32(s, cnt, src, dst);
    else
      convert_f32_to_f64(s, cnt, src, dst);
  }
  template <typename S>
  void out(int64_t cnt, const T* src, S* dst) {
    if constexpr (sizeof(S) == sizeof(T))
      CUCHK(cudaMemcpyAsync(dst, src, sizeof(T) * cnt, cudaMemcpyDeviceToDevice, s));
    else if constexpr (sizeof(T) == 4)
      convert_f32_to_f64(s, cnt, src, dst);
    else
      convert_f64_to_f32(s, cnt, src, dst);
  }
  void solve(phsvds_ctx* ctx, int q, double* Tb, const double* Xu, const double* theta, const double* Xl, int nl,
             const double* dC = nullptr, double guard = 0.0) override {
    run(ctx, q, Tb, Xu, theta, Xl, nl, dC, guard);
  }
  void solve(phsvds_ctx* ctx, int q, float* Tb, const float* Xu, const double* theta, const float* Xl, int nl,
             const double* dC = nullptr, double guard = 0.0) override {
    run(ctx, q, Tb, Xu, theta, Xl, nl, dC, guard);
  }
  template <typename S>
  void run(phsvds_ctx* ctx, int q, S* Tb, const S* Xu, const double* theta, const S* Xl, int nl, const double* dC,
           double guard) {
    Host h(ctx);
    const size_t nq = (size_t)n * q;
    const bool scaled = dC != nullptr;
    in((int64_t)nq, Tb, R);
    in((int64_t)nq, Xu, X);
    if (nl) in((int64_t)n * nl, Xl, Xq);
    // the scaled form projects against Q = [Xl, X]
    const int nq_ = scaled ? nl + q : nl;
    if (scaled) {
      CUCHK(cudaMemcpyAsync(Xq + (size_t)n * nl, X, sizeof(T) * nq, cudaMemcpyDeviceToDevice, s));
      jd_dscale<T>(s, n, dC, guard, ds);
      jd_rowscale<T>(s, n, q, ds, R, R);
    }
    zero(s, v, (size_t)n * 8);   // the columns past q feed the SpMM's padding
    if (scaled) zero(s, U, (size_t)n * 8);
    zero(s, acc, 32);
    jd_colnorms<T>(s, n, q, R, acc);
    jd_init<T>(s, n, q, R, r1, r2, v, sol, w1, w2, acc, sc);
    const int w = spmm_width(q);
    const size_t nacc = 32 + (size_t)8 * nq_;
    Basis<T> P{Xq, n, nq_, nullptr, 0, 0};
    // u: the operator's input (v, or P D^{-1/2} v in the scaled form)
    T* u = scaled ? U : v;
    auto step = [&]() {
      if (scaled) {
        jd_rowscale<T>(s, n, q, ds, v, U);
        zero(s, g1, (size_t)nq_ * q);
        cgs_pass<T>(s, n, P, U, n, q, nullptr, g1, nullptr);
        cgs_pass<T>(s, n, P, U, n, q, g1, nullptr, nullptr);
      }
      cm_to_rm<T>(s, n, u, n, w, Xrm);
      op.apply(s, w, Xrm, Yrm);
      rm_to_cm<T>(s, n, Yrm, w, Cv, n);
      zero(s, acc, nacc);
      if (nq_) cgs_pass<T>(s, n, P, Cv, n, q, nullptr, acc + 32, nullptr);
      jd_dots<T>(s, n, q, u, X, Cv, acc);
      jd_step<T>(s, n, q, nq_, Cv, v, u, scaled ? nullptr : X, Xq, theta, scaled ? ds : nullptr, r1, r2, w1, w2, sol,
                 acc, sc, tol);
    };
    double* hact = h.at<double>(16384);  // bytes [16384, 16448)
    int it = 0;
    while (it < maxit) {
      const int m = std::min(chunk, maxit - it);
      graphs.run(s, (3ull << 40) | ((uint64_t)scaled << 32) | ((uint64_t)m << 16) | ((uint64_t)nq_ << 8) | (uint64_t)q,
                 [&]() {
        for (int i = 0; i < m; ++i) step();
      });
      it += m;
      CUCHK(cudaMemcpyAsync(hact, sc + JD_FIELD_ACT * 8, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
      sync(s);
      bool any = false;
      for (int c = 0; c < q; ++c) any = any || hact[c] != 0.0;
      if (!any) break;
    }
    steps += it;
    ++solves;
    if (scaled) jd_rowscale<T>(s, n, q, ds, sol, sol);
    out((int64_t)nq, sol, Tb);
  }
};

struct Stage1Out {
  std::vector<double> lam;   // k eigenvalues of C (target order)
  double theta_max = 0.0;
  int64_t iters = 0, restarts = 0, mv = 0;
  int64_t jac_sweeps = 0, jac_rot = 0, jac_calls = 0, jac_dim = 0;
  int fell_back = 0;
  int64_t fell_back_at = 0, recorded = 0, stag_locks = 0;
};

// Device state of the learned correction (PHSVDS_PREC_LEARNED) for one solve.
struct LearnedDev {
  const float* feat = nullptr;  // 3 planes of n floats
  int nx = 0, ny = 0;
  float *wf = nullptr, *wt = nullptr, *xin = nullptr, *a1 = nullptr, *a2 = nullptr, *yout = nullptr;
  double* nrm2 = nullptr;
  int stall_window = 0;
};

// A preconditioner P ~ B^{-1} of Sec. 4 applied in the Olsen form (stage 2 and
// the B runs of Algorithm 3): mode 1 [0 A M; M A^T 0] with M = diag(C)^{-1}
// (pd = diag(C), |d| below pguard raised), mode 2 [0 M^{-1}; M^{-T} 0] from a
// given diagonal M ~ A (pd = M, square A); vectors in the [v; u] order.
struct BPrecond {
  cudaStream_t s;
  const DevA* A;
  int mode = 0;
  const double* pd = nullptr;
  double pguard = 0.0;
  double *Pr = nullptr, *Px = nullptr, *ptmp = nullptr, *pdots = nullptr;
  void init(cudaStream_t st, Pool& pool, const DevA& a, int md, const double* d, double guard) {
    s = st;
    A = &a;
    mode = md;
    pd = d;
    pguard = guard;
    const size_t N = (size_t)a.m + a.n;
    Pr = pool.get<double>(N);
    Px = pool.get<double>(N);
    ptmp = pool.get<double>((size_t)a.n);
    pdots = pool.get<double>(2);
  }
  void apply(const double* y, double* Py) {
    const int n = A->n;
    if (mode == 1) {  // [M A^T y_u; A M y_v]
      csr_spmm<double>(s, A->At64, 1, y + n, ptmp);
      diag_div(s, n, ptmp, pd, pguard, Py);
      diag_div(s, n, y, pd, pguard, ptmp);
      csr_spmm<double>(s, A->A64, 1, ptmp, Py + n);
    } else {           // [M^{-1} y_u; M^{-T} y_v] (m = n)
      diag_div(s, n, y + n, pd, 0.0, Py);
      diag_div(s, n, y, pd, 0.0, Py + n);
    }
  }
  // t = P r - (x^T P r / x^T P x) P x
  void olsen(const double* r, const double* x, double* t) {
    const int64_t N = (int64_t)A->m + A->n;
    apply(r, Pr);
    apply(x, Px);
    zero(s, pdots, 2);
    dot_accum(s, N, x, Pr, pdots);
    dot_accum(s, N, x, Px, pdots + 1);
    olsen_combine(s, N, Pr, Px, pdots, t);
  }
};

template <typename T, typename Op = COp<T>>
struct Stage1 {
  phsvds_ctx* ctx;
  cudaStream_t s;
  Pool& pool;
  int n, k, b, maxb, mins, kp;
  bool largest;
  double delta, floor_eps;
  int precond;
  const double* diagC;
  Op op;
  uint64_t seed;
  int max_restarts;
  double time_limit_s;
  bool cluster_eig;
  int eig_mode = 0;
  bool eig32_ok = false;  // the last targets are resolvable in FP32 (>= EIG32_GATE theta_max)
  GraphCache graphs;
  std::chrono::steady_clock::time_point t0;
  // device
  T *V, *W, *Xl, *Tb, *Xrm, *Yrm, *Xr, *Rr, *XU;
  double *Aw, *S, *Ht, *w1, *w2, *Sf, *theta, *Hn, *G1, *G2, *P1, *P2, *M1, *M2, *innorm, *norms, *Scols, *thcols,
      *Yt, *A2, *cand, *excl, *sprev, *dots, *thU;
  int *order, *flags, *jn, *idx;
  // host state
  int j = 0, nlock = 0, nsp = 0, rand_ctr = 0;
  bool s_ident = true;
  Stage1Out out;
  // learned correction: stall watch (progress = a lock or a halved smallest
  // target residual within stall_window iterations)
  const LearnedDev* lp = nullptr;
  int64_t stall_it0 = 0;
  double stall_best = 0.0;
  int stall_locks = -1;
  // stagnation watch of the stage-1 targets
  double stag_best = INFINITY;
  int64_t stag_it = 0;
  int stag_window = 50;
  // residual recording (FP64 pass only)
  double* rec_r = nullptr;
  int rec_max = 0, rec_every = 0;
  // Jacobi-Davidson corrections with FP32 inner solves (FP64 continuation of
  // the mixed-precision stage 1), or null for the plain GD+k correction
  InnerSolver* jd = nullptr;
  // the Olsen correction with a shift-free M (a preconditioner given by the
  // caller, M^{-1} M^{-T} of Sec. 4): diagC holds m_j^2 and theta is taken as 0
  bool shift_free = false;
  // GD+k on B (the B runs of Algorithm 3): targets are the positive
  // eigenvalues nearest zero (those above 1e-12 of the largest magnitude, so
  // that the m - n zero eigenvalues of a rectangular A are not taken), a pair
  // converges at ||r|| < delta ||A|| / sqrt(2), ||A|| the largest |theta| seen,
  // and bp (if set) corrects in the Olsen form with a preconditioner of B
  bool bmode = false;
  BPrecond* bp = nullptr;
  // bounded runs (Algorithm 3): stop after stop_after iterations (0: run to
  // convergence) with partial = true and Xpart = the k current
  // approximations (locked ones first, then the best unconverged Ritz
  // vectors in target order); history = ||r|| of the first unconverged
  // target at every iteration
  int64_t stop_after = 0;
  bool partial = false;
  T* Xpart = nullptr;
  std::vector<double> history;

  Stage1(phsvds_ctx* c, Pool& p, int n_, int k_, const phsvds_opts& o, bool largest_, double delta_, double eps,
         int precond_, const double* diag, Op op_)
      : ctx(c), s(c->stream), pool(p), n(n_), k(k_), largest(largest_), delta(delta_), precond(precond_),
        diagC(diag), op(op_) {
    b = std::max(1, std::min(o.block_size, k));
    maxb = o.max_basis;
    mins = o.min_restart;
    kp = b;
    floor_eps = o.eps_factor * eps;
    seed = o.seed;
    max_restarts = o.max_restarts;
    time_limit_s = o.time_limit_s;
    cluster_eig = o.projected_solver != 1;
    eig_mode = o.projected_solver;
    graphs.enabled = !o.profile;  // the per-class timing events are not captured
    stag_window = std::max(100, 6 * (maxb - mins));
    const size_t nn = (size_t)n;
    V = pool.get<T>(nn * maxb);
    W = pool.get<T>(nn * maxb);
    Xl = pool.get<T>(nn * k);
    Tb = pool.get<T>(nn * 8);
    Xrm = pool.get<T>(nn * 8);
    Yrm = pool.get<T>(nn * 8);
    Xr = pool.get<T>(nn * 8);
    Rr = pool.get<T>(nn * 8);
    XU = pool.get<T>(nn * 8);
    Aw = pool.get<double>(LD * LD);
    S = pool.get<double>(LD * LD);
    Ht = pool.get<double>(LD * LD);
    w1 = pool.get<double>(LD * LD);
    w2 = pool.get<double>(LD * LD);
    Sf = pool.get<double>(LD * LD);
    theta = pool.get<double>(LD);
    Hn = pool.get<double>(LD * 8);
    G1 = pool.get<double>(LD * 8 + LD);
    G2 = pool.get<double>(LD * 8 + LD);
    P1 = pool.get<double>(64);
    P2 = pool.get<double>(64);
    M1 = pool.get<double>(64);
    M2 = pool.get<double>(64);
    innorm = pool.get<double>(8);
    norms = pool.get<double>(8);
    Scols = pool.get<double>(LD * LD);
    thcols = pool.get<double>(LD);
    Yt = pool.get<double>(LD * LD);
    A2 = pool.get<double>(LD * LD);
    cand = pool.get<double>(LD * (LD + 8));
    excl = pool.get<double>(LD * 8);
    sprev = pool.get<double>(LD * 8);
    dots = pool.get<double>(16);
    thU = pool.get<double>(8);
    order = pool.get<int>(LD);
    flags = pool.get<int>(48);
    jn = pool.get<int>(4);
    idx = pool.get<int>(2 * LD);
    zero(s, sprev, LD * 8);
    zero(s, flags, 48);
  }

  void check_time() {
    if (time_limit_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > time_limit_s) throw PhError{PHSVDS_ERR_TIMEOUT, "time limit reached in stage 1"};
    }
  }

  // Orthonormalise nb (<= 8) columns of Tb against [Xl | V] (classical
  // Gram-Schmidt twice, then CholQR twice) and append them to V.
  void orth_append(int nb) {
    Host h(ctx);
    Basis<T> P{Xl, n, nlock, V, n, j};
    const int p = P.cols();
    for (int attempt = 0;; ++attempt) {
      // two CGS passes against [locked, basis], the Gram of the remainder and
      // its Cholesky (graph-cached: one segment without host syncs).  The
      // second pass is never skipped: one pass leaves the block orthogonal
      // only to the accuracy of its projections, whose per-thread partial
      // sums run over tens of terms (~30 eps), which in FP32 is above the
      // stage's own tolerance.
      auto pass = [&]() {
        zero(s, innorm, nb);
        col_norms2_dense<T>(s, n, Tb, n, nb, innorm);
        zero(s, G1, (size_t)p * nb);
        zero(s, G2, (size_t)p * nb);
        zero(s, P1, (size_t)nb * nb);
        cgs_pass<T>(s, n, P, Tb, n, nb, nullptr, G1, nullptr);
        cgs_pass<T>(s, n, P, Tb, n, nb, G1, G2, nullptr);
        cgs_pass<T>(s, n, P, Tb, n, nb, G2, nullptr, P1);
        chol_factor(s, nb, P1, innorm, 1e-10, M1, flags);
        CUCHK(cudaMemcpyAsync(h.at<int>(0), flags, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost, s));
      };
      graphs.run(s, (1ull << 40) | ((uint64_t)nb << 8) | (uint64_t)nlock << 16 | (uint64_t)j, pass);
      sync(s);
      int* f = h.at<int>(0);
      if (!f[nb]) break;
      if (attempt >= 3) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 1: cannot extend the basis"};
      for (int c = 0; c < nb; ++c)
        if (f[c]) fill_random<T>(s, n, Tb + (size_t)c * n, seed, RS_BREAK + (uint64_t)(rand_ctr++));
    }
  }

  // The accepted block, orthonormalised (CholQR, twice for nb > 1), into V.
  void orth_scale(int nb) {
    if (nb == 1) {
      scale_block<T>(s, n, Tb, n, 1, M1, V + (size_t)j * n, n);
    } else {
      scale_block<T>(s, n, Tb, n, nb, M1, nullptr, 0);
      zero(s, P2, (size_t)nb * nb);
      Basis<T> none{};
      cgs_pass<T>(s, n, none, Tb, n, nb, nullptr, nullptr, P2);
      chol_factor(s, nb, P2, nullptr, 0.0, M2, flags + 8);
      scale_block<T>(s, n, Tb, n, nb, M2, V + (size_t)j * n, n);
    }
  }

  // W(:, j0:j0+nb) = C V(:, j0:j0+nb) in row-major chunks of 8/4/2/1.
  void apply_C(int j0, int nb) {
    int c = 0;
    while (c < nb) {
      const int w = spmm_width(nb - c);
      cm_to_rm<T>(s, n, V + (size_t)(j0 + c) * n, n, w, Xrm);
      op.apply(s, w, Xrm, Yrm);
      rm_to_cm<T>(s, n, Yrm, w, W + (size_t)(j0 + c) * n, n);
      c += w;
    }
  }

  // Append nb columns (already in Tb) to the basis and the Jacobi frame.
  void expand(int nb) {
    orth_append(nb);
    // W's new columns, the new Gram column of H and the frame append: one
    // segment without host syncs (graph-cached)
    auto tail = [&]() {
      orth_scale(nb);
      apply_C(j, nb);
      zero(s, Hn, (size_t)(j + nb) * nb);
      Basis<T> Pv{V, n, j + nb, nullptr, 0, 0};
      cgs_pass<T>(s, n, Pv, W + (size_t)j * n, n, nb, nullptr, Hn, nullptr);
      h_append(s, j, nb, Ht, LD, S, LD, Hn);
      if (nsp) CUCHK(cudaMemset2DAsync(sprev + j, LD * sizeof(double), 0, nb * sizeof(double), nsp, s));
    };
    graphs.run(s, (2ull << 40) | ((uint64_t)nsp << 24) | ((uint64_t)nb << 8) | (uint64_t)j, tail);
    out.mv += nb;
    j += nb;
  }

  // Append more than 8 columns (initial guesses) in chunks.
  void expand_many(const T* X0, int ncol) {
    int c = 0;
    while (c < ncol) {
      const int nb = std::min(8, ncol - c);
      CUCHK(cudaMemcpyAsync(Tb, X0 + (size_t)c * n, sizeof(T) * (size_t)n * nb, cudaMemcpyDeviceToDevice, s));
      expand(nb);
      c += nb;
    }
  }

  double tol_of(double th, double thmax) const {
    if (bmode) return delta * thmax / std::sqrt(2.0);
    const double si = std::sqrt(std::max(th, 0.0)), sn = std::sqrt(std::max(thmax, 0.0));
    return std::max(delta * si * sn, floor_eps * thmax);
  }

  // Runs GD+k to convergence.  X0 (n x nx, may be null) replaces the default
  // start (ones(n,1)/sqrt(n) plus random columns).  On return Xl holds the k
  // locked eigenvectors in target order and V/S/order describe the final basis.
  void run(const T* X0, int nx) {
    t0 = std::chrono::steady_clock::now();
    Host h(ctx);
    if (X0 && nx > 0) {
      expand_many(X0, nx);
    } else {
      fill_const<T>(s, n, (T)(1.0 / std::sqrt((double)n)), Tb);
      for (int c = 1; c < b; ++c) fill_random<T>(s, n, Tb + (size_t)c * n, seed, RS_INIT + c);
      expand(b);
    }
    std::vector<double> thv(LD);
    std::vector<int> ord(LD);
    int nb = 0;
    while (true) {
      check_time();
      if (nb > 0) expand(nb);
      // projected eigensolve: an FP32 bulk pass and an FP64 clean-up of the
      // target pairs when the targets are resolvable in FP32, else FP64
      // Jacobi throughout (GB300's FP64 latency is ~14x its FP32 latency)
      const bool mixed_eig = !bmode && eig_mode == 2 && (largest || eig32_ok);
      const int ntg = bmode ? 0 : std::min(b, k - nlock) + 1;   // B: every pair to the tight threshold
      const int omode = bmode ? 3 : (largest ? 1 : 0);
      const int nt = std::min(std::min(b, k - nlock), j);
      const bool sid = s_ident;
      double* hth = h.at<double>(0);        // bytes [0, 512)
      int* hord = h.at<int>(512);            // bytes [512, 768)
      double* hn = h.at<double>(768);        // bytes [768, 832)
      // projected eigensolve, Ritz vectors and residuals, readbacks: one
      // segment without host syncs, replayed as a cached graph
      auto segment = [&]() {
        if (mixed_eig) {
          eig_mixed(s, j, Ht, S, Aw, Sf, theta, w1, w2, sid, true, ntg, largest ? 1 : 0, 0.0, flags + 16, JAC_REL32,
                    true);
        } else {
          frame_from_true(s, j, Ht, S, Aw, w1, w2, sid ? -1 : 1);
          (cluster_eig ? jacobi_eig_cluster_ld : jacobi_eig_fast_ld)(s, j, Aw, LD, S, LD, theta, JAC_TOL, 60,
                                                                     flags + 12, JAC_REL, ntg, largest ? 1 : 0, 0.0,
                                                                     flags + 13);
        }
        order_theta(s, j, theta, omode, 0.0, order);
        gather_cols(s, j, S, LD, order, nt, Scols, LD, theta, thcols, flags + 14);
        tall_times_small<T>(s, n, V, n, j, Scols, LD, nt, Xr, n, nullptr, 0, nullptr, nullptr);
        zero(s, norms, nt);
        tall_times_small<T>(s, n, W, n, j, Scols, LD, nt, Rr, n, Xr, n, thcols, norms);
        CUCHK(cudaMemcpyAsync(hth, theta, sizeof(double) * j, cudaMemcpyDeviceToHost, s));
        CUCHK(cudaMemcpyAsync(hord, order, sizeof(int) * j, cudaMemcpyDeviceToHost, s));
        CUCHK(cudaMemcpyAsync(hn, norms, sizeof(double) * nt, cudaMemcpyDeviceToHost, s));
        CUCHK(cudaMemcpyAsync(h.at<int>(960), flags + 12, sizeof(int) * 8, cudaMemcpyDeviceToHost, s));
      };
      const uint64_t key = (uint64_t)j | ((uint64_t)nt << 8) | ((uint64_t)ntg << 16) | ((uint64_t)mixed_eig << 24) |
                           ((uint64_t)sid << 25) | ((uint64_t)bmode << 26);
      graphs.run(s, key, segment);
      s_ident = false;
      sync(s);
      out.iters++;
      if (*h.at<int>(968)) throw PhError{PHSVDS_ERR_NAN, "stage 1: corrupted ordering of the Ritz values"};
      if (mixed_eig) {  // FP32 pass + FP64 clean-up
        out.jac_sweeps += *h.at<int>(976) + *h.at<int>(984);
        out.jac_rot += *h.at<int>(980) + *h.at<int>(988);
      } else {
        out.jac_sweeps += *h.at<int>(960);
        out.jac_rot += *h.at<int>(964);
      }
      out.jac_calls += 1;
      out.jac_dim += j;
      for (int i = 0; i < j; ++i) {
        ord[i] = hord[i];
        thv[i] = hth[hord[i]];
        if (!std::isfinite(thv[i])) throw PhError{PHSVDS_ERR_NAN, "stage 1: non-finite Ritz value"};
        out.theta_max = std::max(out.theta_max, bmode ? std::fabs(thv[i]) : thv[i]);
      }
      {
        // the FP32-first projected solve resolves eigenvalues to ~1e-7 theta_max:
        // allowed next iteration only if the coming targets sit well above that
        const int nx = std::min(std::min(b, k - nlock) + 1, j);
        double tmin = INFINITY;
        for (int i = 0; i < nx; ++i) tmin = std::min(tmin, std::fabs(thv[i]));
        eig32_ok = tmin >= EIG32_GATE * out.theta_max;
      }
      std::vector<int> conv, unconv;
      double best_ratio = INFINITY;
      int best_t = -1;
      for (int t = 0; t < nt; ++t) {
        const double rn = std::sqrt(std::max(hn[t], 0.0));
        if (!std::isfinite(rn)) throw PhError{PHSVDS_ERR_NAN, "stage 1: non-finite residual"};
        const double tl = tol_of(thv[t], out.theta_max);
        (rn < tl ? conv : unconv).push_back(t);
        if (rn >= tl && rn / tl < best_ratio) best_ratio = rn / tl, best_t = t;
      }
      // Stage 1 stops at the accuracy it can attain (Sec. 3.1): a target whose
      // residual has stopped halving sits on the rounding floor of the
      // products with C -- within STAG_NEAR of its tolerance for a window of
      // iterations, or within STAG_RATIO for STAG_LONG iterations; it is
      // locked, and the switch test hands it to stage 2.
      if (!conv.empty() || best_t < 0) {
        stag_best = INFINITY;
        stag_it = out.iters;
      } else if (best_ratio < 0.5 * stag_best) {
        stag_best = best_ratio;
        stag_it = out.iters;
      } else if ((best_ratio < STAG_NEAR && out.iters - stag_it >= stag_window) ||
                 (best_ratio < STAG_RATIO && out.iters - stag_it >= STAG_LONG)) {
        conv.push_back(best_t);
        unconv.erase(std::find(unconv.begin(), unconv.end(), best_t));
        ++out.stag_locks;
        stag_best = INFINITY;
        stag_it = out.iters;
      }
      if (!unconv.empty()) history.push_back(std::sqrt(std::max(hn[unconv[0]], 0.0)));
      if (trace_on())
        fprintf(stderr, "s1[%d] it=%lld j=%d nlock=%d th0=%.17g rn0=%.6e thmax=%.6e nconv=%d\n", (int)sizeof(T),
                (long long)out.iters, j, nlock, thv[0], std::sqrt(std::max(hn[0], 0.0)), out.theta_max,
                (int)conv.size());
      if (rec_r && rec_every > 0 && out.recorded < rec_max && out.iters % rec_every == 0 && nt > 0) {
        if constexpr (sizeof(T) == 8) {
          CUCHK(cudaMemcpyAsync(rec_r + (size_t)out.recorded * n, Rr, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
          sync(s);
          ++out.recorded;
        }
      }
      if (precond == PHSVDS_PREC_LEARNED && lp && lp->stall_window > 0 && nt > 0) {
        double cur = INFINITY;
        for (int t = 0; t < nt; ++t) cur = std::min(cur, std::sqrt(std::max(hn[t], 0.0)));
        if (nlock + (int)conv.size() > stall_locks || cur < 0.5 * stall_best) {
          stall_locks = nlock + (int)conv.size();
          stall_best = cur;
          stall_it0 = out.iters;
        } else if (out.iters - stall_it0 >= lp->stall_window) {
          precond = diagC ? PHSVDS_PREC_JACOBI : PHSVDS_PREC_NONE;
          out.fell_back = 1;
          out.fell_back_at = out.iters;
        }
      }
      for (int t : conv) {
        CUCHK(cudaMemcpyAsync(Xl + (size_t)nlock * n, Xr + (size_t)t * n, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
        out.lam.push_back(thv[t]);
        ++nlock;
      }
      if (nlock >= k) {
        final_conv = conv;
        final_ord = ord;
        return;
      }
      if (stop_after > 0 && out.iters >= stop_after) {
        // the k current approximations: locked first, then the best
        // unconverged Ritz vectors in target order
        partial = true;
        Xpart = pool.get<T>((size_t)n * k);
        if (nlock) CUCHK(cudaMemcpyAsync(Xpart, Xl, sizeof(T) * (size_t)n * nlock, cudaMemcpyDeviceToDevice, s));
        int* hi = h.at<int>(2048);
        int nf = 0;
        for (int i = 0; i < j && nf < k - nlock; ++i)
          if (std::find(conv.begin(), conv.end(), i) == conv.end()) hi[nf++] = ord[i];
        CUCHK(cudaMemcpyAsync(idx, hi, sizeof(int) * nf, cudaMemcpyHostToDevice, s));
        gather_cols(s, j, S, LD, idx, nf, cand, LD, nullptr, nullptr);
        tall_times_small<T>(s, n, V, n, j, cand, LD, nf, Xpart + (size_t)nlock * n, n, nullptr, 0, nullptr, nullptr);
        sync(s);
        return;
      }
      // frame indices kept (sorted order), excluding the converged targets
      std::vector<int> keep;
      for (int i = 0; i < j; ++i)
        if (std::find(conv.begin(), conv.end(), i) == conv.end()) keep.push_back(ord[i]);
      const bool restart = (int)keep.size() + (int)unconv.size() > maxb;
      const int nu = (int)unconv.size();
      // corrections first (X/R columns of the unconverged targets into XU / Tb)
      for (int c = 0; c < nu; ++c) {
        CUCHK(cudaMemcpyAsync(Tb + (size_t)c * n, Rr + (size_t)unconv[c] * n, sizeof(T) * n,
                              cudaMemcpyDeviceToDevice, s));
        if (precond == PHSVDS_PREC_JACOBI || jd)
          CUCHK(cudaMemcpyAsync(XU + (size_t)c * n, Xr + (size_t)unconv[c] * n, sizeof(T) * n,
                                cudaMemcpyDeviceToDevice, s));
      }
      if (jd && nu > 0) {
        double* hu = h.at<double>(1152);   // bytes [1152, 1216): theta of the corrected columns
        for (int c = 0; c < nu; ++c) hu[c] = thv[unconv[c]];
        CUCHK(cudaMemcpyAsync(thU, hu, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        if (precond == PHSVDS_PREC_JACOBI)
          jd->solve(ctx, nu, Tb, XU, thU, Xl, nlock, diagC, EPS64 * std::max(out.theta_max, 1e-300));
        else
          jd->solve(ctx, nu, Tb, XU, thU, Xl, nlock);
      }
      if (precond == PHSVDS_PREC_LEARNED && lp && nu > 0) {
        double* hu2 = h.at<double>(1088);    // bytes [1088, 1152): ||r||^2 of the corrected columns
        for (int c = 0; c < nu; ++c) hu2[c] = std::max(hn[unconv[c]], 0.0);
        CUCHK(cudaMemcpyAsync(lp->nrm2, hu2, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        cnn_pack<T>(s, n, nu, Tb, n, lp->nrm2, lp->feat, lp->xin);
        cnn_forward(s, nu, lp->nx, lp->ny, lp->wf, lp->xin, lp->a1, lp->a2, lp->yout);
        cnn_unpack<T>(s, n, nu, lp->yout, Tb, n);
      }
      if constexpr (sizeof(T) == 8) {
        if (bp && nu > 0)
          for (int c = 0; c < nu; ++c) bp->olsen(Tb + (size_t)c * n, Xr + (size_t)unconv[c] * n, Tb + (size_t)c * n);
      }
      if (precond == PHSVDS_PREC_JACOBI && !jd && nu > 0) {
        double* hu = h.at<double>(1024);     // bytes [1024, 1088)
        for (int c = 0; c < nu; ++c) hu[c] = shift_free ? 0.0 : thv[unconv[c]];
        CUCHK(cudaMemcpyAsync(thU, hu, sizeof(double) * nu, cudaMemcpyHostToDevice, s));
        zero(s, dots, 2 * nu);
        const double guard = EPS64 * std::max(out.theta_max, 1e-300);
        jacobi_dots<T>(s, n, diagC, XU, n, Tb, n, nu, thU, guard, dots);
        jacobi_apply<T>(s, n, diagC, XU, n, Tb, n, nu, thU, guard, dots, Tb, n);
      }
      if (restart || !conv.empty()) {
        if (restart && ++out.restarts > max_restarts)
          throw PhError{PHSVDS_ERR_NOT_CONVERGED, "stage 1: restart limit reached"};
        int* hi = h.at<int>(2048);           // bytes [2048, 2560)
        const int nkeep = (int)keep.size();
        for (int i = 0; i < nkeep; ++i) hi[i] = keep[i];
        for (size_t i = 0; i < conv.size(); ++i) hi[LD + i] = ord[conv[i]];
        CUCHK(cudaMemcpyAsync(idx, hi, sizeof(int) * 2 * LD, cudaMemcpyHostToDevice, s));
        gather_cols(s, j, S, LD, idx, nkeep, cand, LD, nullptr, nullptr);
        int nc = nkeep, lim_a = nkeep, nmax = nkeep;
        if (restart) {
          lim_a = std::min(nkeep, mins - kp);
          nmax = mins;
          if (nsp) {
            CUCHK(cudaMemcpy2DAsync(cand + (size_t)nkeep * LD, LD * sizeof(double), sprev, LD * sizeof(double),
                                    j * sizeof(double), nsp, cudaMemcpyDeviceToDevice, s));
            nc += nsp;
          }
        }
        const int ne = (int)conv.size();
        if (ne) gather_cols(s, j, S, LD, idx + LD, ne, excl, LD, nullptr, nullptr);
        build_transform(s, j, S, LD, Aw, LD, cand, LD, nc, nkeep, lim_a, 1, excl, LD, ne, nmax, Yt, LD, jn, nullptr,
                        LD);
        int jnew = nkeep;
        if (restart) {
          CUCHK(cudaMemcpyAsync(h.at<int>(12288), jn, sizeof(int), cudaMemcpyDeviceToHost, s));
          sync(s);
          jnew = *h.at<int>(12288);
          if (jnew < 1 || jnew > maxb) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 1: restart basis size out of range"};
        }
        tall_times_small<T>(s, n, V, n, j, Yt, LD, jnew, V, n, nullptr, 0, nullptr, nullptr);
        if (restart && out.restarts % W_REFRESH == 0) {
          apply_C(0, jnew);  // W = C V afresh: W <- W Y drifts from C V by rounding at every restart
          out.mv += jnew;
        }
        else
          tall_times_small<T>(s, n, W, n, j, Yt, LD, jnew, W, n, nullptr, 0, nullptr, nullptr);
        gram_full<T>(s, n, V, W, jnew, Ht, w1);
        set_identity(s, jnew, S, LD);
        s_ident = true;
        j = jnew;
        // the unconverged targets are the first nu columns of the new basis
        double* hs = h.at<double>(4096);     // bytes [4096, 8192)
        for (int c = 0; c < nu; ++c)
          for (int r = 0; r < LD; ++r) hs[r + c * LD] = (r == c) ? 1.0 : 0.0;
        if (nu) CUCHK(cudaMemcpyAsync(sprev, hs, sizeof(double) * LD * nu, cudaMemcpyHostToDevice, s));
        nsp = nu;
      } else {
        // +k vectors of the next restart: this iteration's target coefficients
        for (int c = 0; c < nu; ++c)
          CUCHK(cudaMemcpyAsync(sprev + (size_t)c * LD, Scols + (size_t)unconv[c] * LD, sizeof(double) * j,
                                cudaMemcpyDeviceToDevice, s));
        nsp = nu;
      }
      nb = nu;
      if (nb == 0 && j == 0) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 1: empty basis"};
    }
  }
  std::vector<int> final_conv, final_ord;
};

// ---------------------------------------------------------------------------
// FP64 helpers shared by the Rayleigh-Ritz post-process and stage 2
// ---------------------------------------------------------------------------
struct F64Ctx {
  phsvds_ctx* ctx;
  cudaStream_t s;
  Pool& pool;
  DevA& A;
  double *t1, *t2, *acc;   // n- and m-sized temporaries, accumulators
  F64Ctx(phsvds_ctx* c, Pool& p, DevA& a) : ctx(c), s(c->stream), pool(p), A(a) {
    t1 = pool.get<double>((size_t)a.m + a.n);
    t2 = pool.get<double>((size_t)a.m + a.n);
    acc = pool.get<double>(64);
  }
  // w = B x, x = [v; u] (n + m)
  void B(const double* x, double* w) {
    csr_spmm<double>(s, A.At64, 1, x + A.n, w);
    csr_spmm<double>(s, A.A64, 1, x, w + A.n);
  }
};

// Orthonormalise one column t (length N) against [P1 | P2] (FP64, CGS twice),
// replacing it by a random vector when it is numerically dependent.  Result
// written to dst.  Returns false if even random replacements fail.
struct Orth1 {
  phsvds_ctx* ctx;
  cudaStream_t s;
  double *G1, *G2, *tn, *inn, *minv;
  uint64_t seed;
  int rand_ctr = 0;
  Orth1(phsvds_ctx* c, Pool& p, uint64_t sd) : ctx(c), s(c->stream), seed(sd) {
    G1 = p.get<double>(2 * LD);
    G2 = p.get<double>(2 * LD);
    tn = p.get<double>(4);
    inn = p.get<double>(4);
    minv = p.get<double>(4);
  }
  // skip_below > 0: a t that keeps at most that fraction of its squared norm
  // is left out (returns false) instead of replaced by a random vector
  double last_kept = 0.0;  // squared norm kept by the last run (relative), for the trace
  bool run(int N, const Basis<double>& P, double* t, double* dst, double skip_below = -1.0) {
    Host h(ctx);
    const int p = P.cols();
    for (int attempt = 0;; ++attempt) {
      zero(s, inn, 1);
      col_norms2_dense<double>(s, N, t, N, 1, inn);
      zero(s, G1, p);
      zero(s, G2, p);
      zero(s, tn, 1);
      cgs_pass<double>(s, N, P, t, N, 1, nullptr, G1, nullptr);
      cgs_pass<double>(s, N, P, t, N, 1, G1, G2, nullptr);
      cgs_pass<double>(s, N, P, t, N, 1, G2, nullptr, tn);
      CUCHK(cudaMemcpyAsync(h.at<double>(0), tn, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUCHK(cudaMemcpyAsync(h.at<double>(8), inn, sizeof(double), cudaMemcpyDeviceToHost, s));
      sync(s);
      const double a = *h.at<double>(0), b0 = *h.at<double>(8);
      last_kept = b0 > 0 ? a / b0 : 0.0;
      if (!std::isfinite(a)) throw PhError{PHSVDS_ERR_NAN, "non-finite vector in orthogonalisation"};
      if (skip_below > 0 && !(a > skip_below * b0)) return false;
      if (b0 > 0 && a > 1e-20 * b0) {
        const double f = 1.0 / std::sqrt(a);
        scal(s, N, f, nullptr, t);
        if (dst != t) CUCHK(cudaMemcpyAsync(dst, t, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        return true;
      }
      if (attempt >= 3) throw PhError{PHSVDS_ERR_BREAKDOWN, "cannot extend the basis"};
      fill_random<double>(s, N, t, seed, RS_BREAK + 0x100000 + (uint64_t)(rand_ctr++));
    }
  }
};

// Rayleigh-Ritz of C on [Xl, extra] (Algorithm 1 step 3), FP64.  Returns the k
// new eigenvalues (target order) and writes the k new vectors to Xout (n x k).
static std::vector<double> rayleigh_ritz_post(phsvds_ctx* ctx, Pool& pool, DevA& A, COp<double>& op, const double* Xl,
                                              int k, const double* Extra, int nextra, bool largest, uint64_t seed,
                                              double* Xout, int64_t& mv) {
  cudaStream_t s = ctx->stream;
  const int n = A.n;
  const int q = k + nextra;
  double* Q = pool.get<double>((size_t)n * q);
  double* WQ = pool.get<double>((size_t)n * q);
  double* Xrm = pool.get<double>((size_t)n * 8);
  double* Yrm = pool.get<double>((size_t)n * 8);
  double* tmp = pool.get<double>(n);
  double* H = pool.get<double>(LD * LD);
  double* Hc = pool.get<double>(LD * 8);
  double* S = pool.get<double>(LD * LD);
  double* th = pool.get<double>(LD);
  double* Sc = pool.get<double>(LD * LD);
  int* ord = pool.get<int>(LD);
  int* sw = pool.get<int>(2);
  Orth1 orth(ctx, pool, seed);
  for (int c = 0; c < q; ++c) {
    const double* src = c < k ? Xl + (size_t)c * n : Extra + (size_t)(c - k) * n;
    CUCHK(cudaMemcpyAsync(tmp, src, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    Basis<double> P{Q, n, c, nullptr, 0, 0};
    orth.run(n, P, tmp, Q + (size_t)c * n);
  }
  for (int c = 0; c < q;) {
    const int w = spmm_width(q - c);
    cm_to_rm<double>(s, n, Q + (size_t)c * n, n, w, Xrm);
    op.apply(s, w, Xrm, Yrm);
    rm_to_cm<double>(s, n, Yrm, w, WQ + (size_t)c * n, n);
    c += w;
  }
  mv += q;
  for (int c = 0; c < q;) {
    const int w = std::min(8, q - c);
    zero(s, Hc, (size_t)q * w);
    Basis<double> P{Q, n, q, nullptr, 0, 0};
    cgs_pass<double>(s, n, P, WQ + (size_t)c * n, n, w, nullptr, Hc, nullptr);
    CUCHK(cudaMemcpy2DAsync(H + (size_t)c * LD, LD * sizeof(double), Hc, q * sizeof(double), q * sizeof(double), w,
                            cudaMemcpyDeviceToDevice, s));
    c += w;
  }
  // symmetrised H into the frame matrix Sc (frame_append with an empty frame
  // expects the new columns compact, ld = q) and S = I
  double* Hq = pool.get<double>((size_t)q * q);
  CUCHK(cudaMemcpy2DAsync(Hq, q * sizeof(double), H, LD * sizeof(double), q * sizeof(double), q,
                          cudaMemcpyDeviceToDevice, s));
  frame_append(s, 0, q, Sc, LD, S, LD, Hq);
  jacobi_eig_cluster_ld(s, q, Sc, LD, S, LD, th, JAC_TOL, 60, sw, JAC_TOL, 0, 0, 0.0, nullptr);
  order_theta(s, q, th, largest ? 1 : 0, 0.0, ord);
  double* Sk = pool.get<double>(LD * LD);
  double* thk = pool.get<double>(LD);
  gather_cols(s, q, S, LD, ord, k, Sk, LD, th, thk);
  tall_times_small<double>(s, n, Q, n, q, Sk, LD, k, Xout, n, nullptr, 0, nullptr, nullptr);
  Host h(ctx);
  CUCHK(cudaMemcpyAsync(h.at<double>(0), thk, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
  sync(s);
  return std::vector<double>(h.at<double>(0), h.at<double>(0) + k);
}

// ---------------------------------------------------------------------------
// Stage 2: refined projection on B (Algorithm 2), FP64
// ---------------------------------------------------------------------------
// The JDQMR correction of stage 2 (Sec. 4): an inexact solution of
// (I - QQ^T)(B - mu I)(I - QQ^T) t = -(I - QQ^T) r, Q = [locked vectors and
// mirrors, x], by MINRES in FP64 with the dynamic stop on the eigen-residual
// of x + t (k_inner.cu), one equation per outer iteration.
struct InnerJD2 {
  cudaStream_t s;
  F64Ctx& f;
  int64_t N;
  int n, maxit, patience, chunk = 10;
  double *R, *r1, *r2, *v, *t, *w1, *w2, *Bv, *Bt, *Bw1, *Bw2, *Bx, *tbest, *acc, *sc, *mu;
  GraphCache graphs;
  int64_t steps = 0, solves = 0;
  InnerJD2(phsvds_ctx* c, Pool& pool, F64Ctx& ff, int maxit_, int patience_, bool use_graphs)
      : s(c->stream), f(ff), N((int64_t)ff.A.m + ff.A.n), n(ff.A.n), maxit(maxit_), patience(patience_) {
    for (double** p : {&R, &r1, &r2, &v, &t, &w1, &w2, &Bv, &Bt, &Bw1, &Bw2, &Bx, &tbest}) *p = pool.get<double>(N);
    acc = pool.get<double>(256);
    sc = pool.get<double>(JD_NSCALAR * 8 + 8);
    mu = pool.get<double>(1);
    graphs.enabled = use_graphs;
  }
  // out = the correction for the refined pair (mu, x) with residual r and
  // B x = Bx_in; Q: nq columns (the last one x).  Returns the steps taken.
  int solve(phsvds_ctx* ctx, const double* Q, int nq, const double* x, const double* Bx_in, double mu_h,
            const double* r, double eta_tol, double* out) {
    Host h(ctx);
    Basis<double> PQ{Q, (int)N, nq, nullptr, 0, 0};
    // right-hand side -(I - QQ^T) r
    CUCHK(cudaMemcpyAsync(R, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    zero(s, acc, 256);
    cgs_pass<double>(s, (int)N, PQ, R, (int)N, 1, nullptr, acc + 32, nullptr);
    cgs_pass<double>(s, (int)N, PQ, R, (int)N, 1, acc + 32, nullptr, nullptr);
    scal(s, N, -1.0, nullptr, R);
    CUCHK(cudaMemcpyAsync(Bx, Bx_in, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    double* hm = h.at<double>(16448);   // bytes [16448, 16456)
    *hm = mu_h;
    CUCHK(cudaMemcpyAsync(mu, hm, sizeof(double), cudaMemcpyHostToDevice, s));
    CUCHK(cudaMemcpyAsync(tbest, r, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    s2_start(s, N, R, r1, r2, v, t, w1, w2, Bt, Bw1, Bw2, acc, sc);
    auto step = [&]() {
      f.B(v, Bv);
      zero(s, acc, 256);
      cgs_pass<double>(s, (int)N, PQ, Bv, (int)N, 1, nullptr, acc + 32, nullptr);
      dot_accum(s, N, v, Bv, acc);
      dot_accum(s, N, v, v, acc + 8);
      s2_step(s, N, nq, Bv, v, Q, mu, r1, r2, w1, w2, t, Bw1, Bw2, Bt, x, Bx, tbest, acc, sc, eta_tol, patience,
              maxit);
    };
    double* hs = h.at<double>(16456);   // bytes [16456, 16472): act, steps
    int it = 0;
    while (it < maxit) {
      const int m = std::min(chunk, maxit - it);
      graphs.run(s, (4ull << 40) | ((uint64_t)m << 16) | (uint64_t)nq, [&]() {
        for (int i = 0; i < m; ++i) step();
      });
      it += m;
      CUCHK(cudaMemcpyAsync(hs, sc + JD_FIELD_ACT * 8, sizeof(double), cudaMemcpyDeviceToHost, s));
      CUCHK(cudaMemcpyAsync(hs + 1, sc + JD2_FIELD_STEPS, sizeof(double), cudaMemcpyDeviceToHost, s));
      sync(s);
      if (hs[0] == 0.0) break;
    }
    const int taken = (int)hs[1];
    steps += taken;
    ++solves;
    CUCHK(cudaMemcpyAsync(out, tbest, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    return taken;
  }
};

struct Stage2 {
  phsvds_ctx* ctx;
  cudaStream_t s;
  Pool& pool;
  F64Ctx& f;
  int m, n, N, k, maxb, mins;
  double delta, normA;
  uint64_t seed;
  int max_restarts;
  double time_limit_s;
  std::chrono::steady_clock::time_point t0;
  double *V, *W, *Q, *Xl, *x0, *tv, *xr, *rr;
  double *Aw, *S, *Ht, *w1, *w2, *Sf, *theta, *R, *s1, *rq, *Hn, *Yt, *cand, *excl,
      *sprev, *nrm, *G1, *G2, *tn2, *minv;
  bool s_ident = true;
  int *order, *sw, *jn;
  Orth1 orth;
  int j = 0, nl = 0;
  int64_t iters = 0, restarts = 0, mv = 0;
  std::vector<double> th_lock;
  // correction operator P of B (Sec. 4) in the Olsen form, or none (t = r)
  BPrecond bpre;
  // deflated vectors: the locked ones, and with the JDQMR correction also the
  // mirror [v; -u] of each locked tiny pair (for sigma <= sqrt(eps) ||A|| the
  // pair +-sigma of B is not separable at the tolerance and both eigenvectors
  // belong to one triplet), with room for x as the last column of Q
  double* D = nullptr;
  int nd = 0;
  InnerJD2* jd2 = nullptr;
  double* Bxr = nullptr;
  // the residual of the current target's own initial guess at its shift (set
  // at each target switch; negative: not measured)
  double guess_res = -1.0;
  int64_t guess_restarts = 0;

  Stage2(phsvds_ctx* c, Pool& p, F64Ctx& ff, DevA& A, int k_, const phsvds_opts& o, double delta_, double normA_)
      : ctx(c), s(c->stream), pool(p), f(ff), m(A.m), n(A.n), N(A.m + A.n), k(k_), maxb(o.max_basis),
        mins(o.min_restart), delta(delta_), normA(normA_), seed(o.seed), max_restarts(o.max_restarts),
        time_limit_s(o.time_limit_s), orth(c, p, o.seed) {
    const size_t NN = (size_t)N;
    V = pool.get<double>(NN * maxb);
    W = pool.get<double>(NN * maxb);
    Q = pool.get<double>(NN * maxb);
    Xl = pool.get<double>(NN * k);
    D = pool.get<double>(NN * (2 * k + 1));
    Bxr = pool.get<double>(NN);
    x0 = pool.get<double>(NN * k);
    tv = pool.get<double>(NN);
    xr = pool.get<double>(NN);
    rr = pool.get<double>(NN);
    Aw = pool.get<double>(LD * LD);
    S = pool.get<double>(LD * LD);
    Ht = pool.get<double>(LD * LD);
    w1 = pool.get<double>(LD * LD);
    w2 = pool.get<double>(LD * LD);
    Sf = pool.get<double>(LD * LD);
    theta = pool.get<double>(LD);
    R = pool.get<double>(LD * LD);
    s1 = pool.get<double>(LD);
    rq = pool.get<double>(4);
    Hn = pool.get<double>(LD);
    Yt = pool.get<double>(LD * LD);
    cand = pool.get<double>(LD * (2 * LD + 2));
    excl = pool.get<double>(LD);
    sprev = pool.get<double>(LD);
    nrm = pool.get<double>(4);
    G1 = pool.get<double>(LD);
    G2 = pool.get<double>(LD);
    tn2 = pool.get<double>(4);
    minv = pool.get<double>(4);
    order = pool.get<int>(LD);
    sw = pool.get<int>(16);
    jn = pool.get<int>(4);
  }

  void check_time() {
    if (time_limit_s > 0) {
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > time_limit_s) throw PhError{PHSVDS_ERR_TIMEOUT, "time limit reached in stage 2"};
    }
  }

  void set_precond(int mode, const double* d, double guard) { bpre.init(s, pool, f.A, mode, d, guard); }

  // The residual of a lock candidate afresh, ||B x - th x|| from a new product
  // (into tv, free here): the estimate W s1 - th V s1 carries the rounding of
  // every transform that W went through, which near eps ||A|| can sit on
  // either side of the tolerance.
  double fresh_resid(double th) { return resid_of(xr, th); }
  double resid_of(const double* x, double th) {
    Host h(ctx);
    f.B(x, tv);
    ++mv;
    axpby(s, N, -th, x, 1.0, tv);
    zero(s, nrm + 1, 1);
    col_norms2_dense<double>(s, N, tv, N, 1, nrm + 1);
    CUCHK(cudaMemcpyAsync(h.at<double>(24), nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    sync(s);
    return std::sqrt(std::max(*h.at<double>(24), 0.0));
  }

  // The basis restarted from one vector (orthonormalised against D): V = [t],
  // W = [B t], H and the QR afresh at the next iteration.
  void restart_from(const double* t0) {
    CUCHK(cudaMemcpyAsync(tv, t0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    j = 0;
    set_identity(s, LD, S, LD);
    s_ident = true;
    append(tv);
  }

  // Append t (orthonormalised against [Xl | V]) as column j; W(:, j) = B v_j;
  // the frame gets the new column of H = V^T W.
  void append(double* t) {
    Basis<double> P{D, N, nd, V, N, j};
    orth.run(N, P, t, V + (size_t)j * N);
    f.B(V + (size_t)j * N, W + (size_t)j * N);
    ++mv;
    zero(s, Hn, j + 1);
    Basis<double> Pv{V, N, j + 1, nullptr, 0, 0};
    cgs_pass<double>(s, N, Pv, W + (size_t)j * N, N, 1, nullptr, Hn, nullptr);
    h_append(s, j, 1, Ht, LD, S, LD, Hn);
    ++j;
  }

  // QR column c of Z = W - shift V into Q(:, c), R(:, c).
  void qr_col(int c, double shift) {
    double* z = Q + (size_t)c * N;
    CUCHK(cudaMemcpyAsync(z, W + (size_t)c * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    axpby(s, N, -shift, V + (size_t)c * N, 1.0, z);
    Basis<double> P{Q, N, c, nullptr, 0, 0};
    zero(s, G1, c + 1);
    zero(s, G2, c + 1);
    zero(s, tn2, 1);
    cgs_pass<double>(s, N, P, z, N, 1, nullptr, G1, nullptr);
    cgs_pass<double>(s, N, P, z, N, 1, G1, G2, nullptr);
    cgs_pass<double>(s, N, P, z, N, 1, G2, nullptr, tn2);
    qr_column(s, c, c ? G1 : nullptr, c ? G2 : nullptr, tn2, R, LD, nullptr, 0, nullptr, 0, minv, 0);
    scal(s, N, 0.0, minv, z);
  }

  void full_qr(double shift) {
    zero(s, R, LD * LD);  // the strictly lower triangle stays zero
    for (int c = 0; c < j; ++c) qr_col(c, shift);
  }

  // Transform the basis by Y (j x jn basis coordinates, from build_transform).
  void transform(int jnew) {
    tall_times_small<double>(s, N, V, N, j, Yt, LD, jnew, V, N, nullptr, 0, nullptr, nullptr);
    tall_times_small<double>(s, N, W, N, j, Yt, LD, jnew, W, N, nullptr, 0, nullptr, nullptr);
    gram_full<double>(s, N, V, W, jnew, Ht, w1);
    set_identity(s, jnew, S, LD);
    s_ident = true;
    j = jnew;
  }

  // The basis made orthonormal against the deflated set D again (after a
  // mirror joined it): each column orthonormalised against D and the columns
  // before it, then W = B V and H = V^T W afresh.
  void reorthonormalise() {
    const int jj = j;
    for (int c = 0; c < jj; ++c) {
      CUCHK(cudaMemcpyAsync(tv, V + (size_t)c * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      Basis<double> P{D, N, nd, V, N, c};
      orth.run(N, P, tv, V + (size_t)c * N);
      f.B(V + (size_t)c * N, W + (size_t)c * N);
      ++mv;
    }
    gram_full<double>(s, N, V, W, jj, Ht, w1);
    set_identity(s, jj, S, LD);
    s_ident = true;
  }

  // sig_s: k shifts (stage-1 values), Vt: n x k FP64 stage-1 right vectors.
  void run(const std::vector<double>& sig_s, const double* Vt) {
    t0 = std::chrono::steady_clock::now();
    Host h(ctx);
    // ---- initial guesses [v; A v / s] / sqrt(2) (Algorithm 2 step 1, Sec. 3.3)
    zero(s, nrm, 2);
    double* hv = h.at<double>(0);
    for (int i = 0; i < k; ++i) {
      double* xi = x0 + (size_t)i * N;
      CUCHK(cudaMemcpyAsync(xi, Vt + (size_t)i * n, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      if (sig_s[i] > std::sqrt(EPS64) * normA) {
        csr_spmm<double>(s, f.A.A64, 1, xi, xi + n);
        ++mv;
      } else {
        fill_random<double>(s, m, xi + n, seed, RS_U + i);
      }
      zero(s, nrm, 2);
      col_norms2_dense<double>(s, n, xi, N, 1, nrm);
      col_norms2_dense<double>(s, m, xi + n, N, 1, nrm + 1);
      CUCHK(cudaMemcpyAsync(hv + 2 * i, nrm, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
      sync(s);
      const double nv = std::sqrt(hv[2 * i]), nu = std::sqrt(hv[2 * i + 1]);
      if (!(nv > 0) || !(nu > 0)) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 2: zero initial guess"};
      scal(s, n, 1.0 / (nv * std::sqrt(2.0)), nullptr, xi);
      scal(s, m, 1.0 / (nu * std::sqrt(2.0)), nullptr, xi + n);
    }
    // ---- initial basis: K_{s-k}(B, x0_1) and the guesses (Algorithm 2 step 2)
    const int qk = std::max(1, mins - k);
    CUCHK(cudaMemcpyAsync(tv, x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    append(tv);
    for (int r = 1; r < qk; ++r) {
      CUCHK(cudaMemcpyAsync(tv, W + (size_t)(j - 1) * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      append(tv);
    }
    const int nguess = std::min(k - 1, maxb - 1 - j);
    for (int i = 1; i <= nguess; ++i) {
      CUCHK(cudaMemcpyAsync(tv, x0 + (size_t)i * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      append(tv);
    }
    int target = 0;
    double shift = sig_s[0];
    bool qr_full = true;
    bool have_prev = false;
    double r0 = -1.0;
    while (true) {
      check_time();
      ++iters;
      if (qr_full) {
        full_qr(shift);
        qr_full = false;
      }
      // refined vector: smallest right singular vector of R (Sec. 3.2)
      refined_inverse(s, j, R, LD, have_prev ? sprev : nullptr, Ht, LD, RI_MAXIT, RI_TAU, s1, rq, sw + 1);
      tall_times_small<double>(s, N, V, N, j, s1, LD, 1, xr, N, nullptr, 0, nullptr, nullptr);
      zero(s, nrm, 1);
      tall_times_small<double>(s, N, W, N, j, s1, LD, 1, rr, N, xr, N, rq, nrm);
      CUCHK(cudaMemcpyAsync(h.at<double>(0), rq, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
      CUCHK(cudaMemcpyAsync(h.at<double>(16), nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
      sync(s);
      const double th1 = *h.at<double>(0);
      const double rn = std::sqrt(std::max(*h.at<double>(16), 0.0));
      if (!std::isfinite(th1) || !std::isfinite(rn)) throw PhError{PHSVDS_ERR_NAN, "stage 2: non-finite residual"};
      if (r0 < 0) {
        r0 = rn;
        // the first iteration of a target: if the kept basis gives a refined
        // residual far above the target's own guess, start from the guess
        if (guess_res > 0 && rn > 10.0 * guess_res && j > 1) {
          restart_from(x0 + (size_t)target * N);
          ++guess_restarts;
          qr_full = true;
          have_prev = false;
          r0 = -1.0;
          guess_res = -1.0;
          continue;
        }
        guess_res = -1.0;
      }
      const double tolB = delta * normA / std::sqrt(2.0);
      // near the tolerance the estimate is checked against a fresh residual
      const double rf = rn < 4.0 * tolB ? fresh_resid(th1) : -1.0;
      if (trace_on()) {
        if (!have_prev) {
          // the smallest singular value of R by the one-sided Jacobi SVD, beside
          // the inverse iteration's (a diagnostic of the trace only)
          double* Rc = pool.get<double>(LD * LD);
          double* Sc = pool.get<double>(LD * LD);
          double* sg = pool.get<double>(LD);
          CUCHK(cudaMemcpyAsync(Rc, R, sizeof(double) * LD * LD, cudaMemcpyDeviceToDevice, s));
          set_identity(s, j, Sc, LD);
          jacobi_svd_ld(s, j, Rc, LD, Sc, LD, sg, 1e-15, 60, nullptr);
          CUCHK(cudaMemcpyAsync(h.at<double>(4096), sg, sizeof(double) * j, cudaMemcpyDeviceToHost, s));
          sync(s);
          double mn = INFINITY;
          for (int i = 0; i < j; ++i) mn = std::min(mn, *h.at<double>(4096 + 8 * i));
          // the invariants the refined search relies on: W = B V, V orthonormal, V orthogonal to D
          double* bv = pool.get<double>((size_t)N);
          double* gv = pool.get<double>((size_t)LD * LD);
          double* gd = pool.get<double>((size_t)LD * (2 * k + 1));
          double* ww = pool.get<double>(1);
          double werr = 0.0;
          for (int c = 0; c < j; ++c) {
            f.B(V + (size_t)c * N, bv);
            axpby(s, N, -1.0, W + (size_t)c * N, 1.0, bv);
            zero(s, ww, 1);
            col_norms2_dense<double>(s, N, bv, N, 1, ww);
            CUCHK(cudaMemcpyAsync(h.at<double>(8192), ww, sizeof(double), cudaMemcpyDeviceToHost, s));
            sync(s);
            werr = std::max(werr, std::sqrt(std::max(*h.at<double>(8192), 0.0)));
          }
          zero(s, gv, (size_t)j * j);
          Basis<double> PV{V, N, j, nullptr, 0, 0};
          cgs_pass<double>(s, N, PV, V, N, std::min(j, 8), nullptr, gv, nullptr);
          double verr = 0.0, derr = 0.0;
          CUCHK(cudaMemcpyAsync(h.at<double>(8192), gv, sizeof(double) * j * std::min(j, 8), cudaMemcpyDeviceToHost, s));
          sync(s);
          for (int c = 0; c < std::min(j, 8); ++c)
            for (int r = 0; r < j; ++r)
              verr = std::max(verr, std::fabs(*h.at<double>(8192 + 8 * (r + c * j)) - (r == c ? 1.0 : 0.0)));
          if (nd > 0) {
            zero(s, gd, (size_t)nd * 8);
            Basis<double> PD{D, N, nd, nullptr, 0, 0};
            cgs_pass<double>(s, N, PD, V, N, std::min(j, 8), nullptr, gd, nullptr);
            CUCHK(cudaMemcpyAsync(h.at<double>(8192), gd, sizeof(double) * nd * std::min(j, 8), cudaMemcpyDeviceToHost,
                                  s));
            sync(s);
            for (int e = 0; e < nd * std::min(j, 8); ++e) derr = std::max(derr, std::fabs(*h.at<double>(8192 + 8 * e)));
          }
          // the guess's coordinates in the basis, s = V^T x0, and ||(W - mu V) s|| / ||s||
          double* sg2 = pool.get<double>(LD);
          double* yv = pool.get<double>((size_t)N);
          double* wy = pool.get<double>((size_t)N);
          zero(s, sg2, LD);
          cgs_pass<double>(s, N, PV, const_cast<double*>(x0 + (size_t)target * N), N, 1, nullptr, sg2, nullptr);
          tall_times_small<double>(s, N, V, N, j, sg2, LD, 1, yv, N, nullptr, 0, nullptr, nullptr);
          tall_times_small<double>(s, N, W, N, j, sg2, LD, 1, wy, N, nullptr, 0, nullptr, nullptr);
          axpby(s, N, -shift, yv, 1.0, wy);
          double* nn2 = pool.get<double>(2);
          zero(s, nn2, 2);
          col_norms2_dense<double>(s, N, wy, N, 1, nn2);
          col_norms2_dense<double>(s, N, yv, N, 1, nn2 + 1);
          CUCHK(cudaMemcpyAsync(h.at<double>(8192), nn2, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
          sync(s);
          const double rs_ = std::sqrt(std::max(*h.at<double>(8192), 0.0)),
                       ys_ = std::sqrt(std::max(*h.at<double>(8200), 0.0));
          fprintf(stderr, "s2 target %d: guess in the basis: ||V V^T x0|| %.6e, its ||(W - mu V) s|| / ||s|| %.3e\n",
                  target, ys_, ys_ > 0 ? rs_ / ys_ : -1.0);
          fprintf(stderr,
                  "s2 target %d first iteration: sigma_min(R) by SVD %.6e, max ||W - B V|| %.3e, "
                  "|V^T V - I| (first 8 cols) %.3e, |D^T V| (first 8 cols) %.3e, j %d, nd %d\n",
                  target, mn, werr, verr, derr, j, nd);
        }
        CUCHK(cudaMemcpyAsync(h.at<int>(40), sw + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        sync(s);
        fprintf(stderr, "s2 it=%lld j=%d target=%d shift=%.17g th1=%.17g rn=%.6e rf=%.6e sigmin=%.6e ri=%d\n",
                (long long)iters, j, target, shift, th1, rn, rf, *h.at<double>(8), *h.at<int>(40));
      }
      if (rf >= 0.0 && rf < tolB) {
        CUCHK(cudaMemcpyAsync(Xl + (size_t)nl * N, xr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        CUCHK(cudaMemcpyAsync(D + (size_t)nd * N, xr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        ++nl;
        ++nd;
        const bool mirror = jd2 && std::fabs(th1) <= std::sqrt(EPS64) * normA;
        if (mirror) {  // [v; -u], orthonormalised against the deflated set, deflated as well
          // (the mirror is orthogonal to x, but to the other tiny locked
          // pairs only as far as their v and u parts are separately
          // orthogonal, i.e. to the accuracy r / gap of the tiny cluster)
          CUCHK(cudaMemcpyAsync(tv, xr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
          scal(s, m, -1.0, nullptr, tv + n);
          Basis<double> P{D, N, nd, nullptr, 0, 0};
          if (orth.run(N, P, tv, D + (size_t)nd * N, 1e-8)) ++nd;   // (already deflated: left out)
        }
        th_lock.push_back(th1);
        ++target;
        if (target >= k) break;
        // drop s1 from the basis: keep an orthonormal basis of its complement
        // (the span of the other right singular vectors of R), built by
        // Gram-Schmidt of the unit vectors against s1
        if (j > 1) {
          set_identity(s, j, cand, LD);
          build_transform(s, j, S, LD, Aw, LD, cand, LD, j, 0, 0, 0, s1, LD, 1, j - 1, Yt, LD, jn, nullptr, LD);
          CUCHK(cudaMemcpyAsync(h.at<int>(12288), jn, sizeof(int), cudaMemcpyDeviceToHost, s));
          sync(s);
          const int nc = *h.at<int>(12288);
          if (nc < 1 || nc > j - 1) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 2: locking complement size out of range"};
          transform(nc);
          if (mirror) reorthonormalise();
        } else {
          j = 0;  // the basis was s1 alone
          s_ident = true;
        }
        CUCHK(cudaMemcpyAsync(tv, x0 + (size_t)target * N, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        append(tv);
        guess_res = resid_of(x0 + (size_t)target * N, sig_s[target]);
        ++mv;
        if (trace_on()) {
          // the guess's own residual ||B x0 - s x0|| at its shift
          const double* xg = x0 + (size_t)target * N;
          f.B(xg, tv);
          axpby(s, N, -sig_s[target], xg, 1.0, tv);
          zero(s, nrm + 1, 1);
          col_norms2_dense<double>(s, N, tv, N, 1, nrm + 1);
          CUCHK(cudaMemcpyAsync(h.at<double>(24), nrm + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
          sync(s);
          fprintf(stderr, "s2 new target %d: guess keeps %.3e of its squared norm, its residual %.3e\n", target,
                  orth.last_kept, std::sqrt(std::max(*h.at<double>(24), 0.0)));
        }
        shift = sig_s[target];
        qr_full = true;
        have_prev = false;
        r0 = -1.0;
        continue;
      }
      if (j >= maxb) {
        if (++restarts > max_restarts) throw PhError{PHSVDS_ERR_NOT_CONVERGED, "stage 2: restart limit reached"};
        // Ritz pairs of H ordered by closeness to the shift (only the
        // restart needs them)
        eig_mixed(s, j, Ht, S, Aw, Sf, theta, w1, w2, s_ident, true, 1, 2, shift, sw + 2);
        s_ident = false;
        order_theta(s, j, theta, 2, shift, order);
        // candidates: s1, Ritz vectors by closeness to the shift, then the previous s1
        CUCHK(cudaMemcpyAsync(cand, s1, sizeof(double) * j, cudaMemcpyDeviceToDevice, s));
        gather_cols(s, j, S, LD, order, j, cand + LD, LD, nullptr, nullptr);
        int nc = j + 1;
        if (have_prev) {
          CUCHK(cudaMemcpyAsync(cand + (size_t)nc * LD, sprev, sizeof(double) * j, cudaMemcpyDeviceToDevice, s));
          ++nc;
        }
        build_transform(s, j, S, LD, Aw, LD, cand, LD, nc, j + 1, mins - 1, 0, excl, LD, 0, mins, Yt, LD, jn, nullptr,
                        LD);
        CUCHK(cudaMemcpyAsync(h.at<int>(12288), jn, sizeof(int), cudaMemcpyDeviceToHost, s));
        sync(s);
        const int jnew = *h.at<int>(12288);
        if (jnew < 1 || jnew > maxb) throw PhError{PHSVDS_ERR_BREAKDOWN, "stage 2: restart basis size out of range"};
        transform(jnew);
        // s1 is the first new basis vector
        double* hs = h.at<double>(10240);    // bytes [10240, 10752)
        for (int r = 0; r < LD; ++r) hs[r] = r == 0 ? 1.0 : 0.0;
        CUCHK(cudaMemcpyAsync(sprev, hs, sizeof(double) * LD, cudaMemcpyHostToDevice, s));
        have_prev = true;
        if (rn < r0) shift = th1;  // Rayleigh quotient of the refined vector (Sec. 3.2)
        qr_full = true;
      } else {
        CUCHK(cudaMemcpyAsync(sprev, s1, sizeof(double) * j, cudaMemcpyDeviceToDevice, s));
        have_prev = true;
      }
      // ---- expand with t = r, its preconditioned Olsen form, or the JDQMR
      // correction
      if (jd2) {
        tall_times_small<double>(s, N, W, N, j, s1, LD, 1, Bxr, N, nullptr, 0, nullptr, nullptr);   // B x
        CUCHK(cudaMemcpyAsync(D + (size_t)nd * N, xr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
        const int taken = jd2->solve(ctx, D, nd + 1, xr, Bxr, th1, rr, delta * normA / std::sqrt(2.0), tv);
        mv += taken;
      } else if (bpre.mode) {
        bpre.olsen(rr, xr, tv);
        if (bpre.mode == 1) mv += 2;   // one product with A and one with A^T for each of P r and P x
      } else {
        CUCHK(cudaMemcpyAsync(tv, rr, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
      }
      append(tv);
      CUCHK(cudaMemsetAsync(sprev + (j - 1), 0, sizeof(double), s));
      if (!qr_full) qr_col(j - 1, shift);
    }
  }
};

// Final triplets from right vectors V (n x k) and, when U != nullptr, left
// vectors U (m x k): normalise, sigma = u^T A v (or ||A v|| with u = A v/||A v||
// when U is null), residual sqrt(||A v - s u||^2 + ||A^T u - s v||^2).
static void final_triplets(phsvds_ctx* ctx, Pool& pool, DevA& A, int k, double* Vd, double* Ud, bool have_u,
                           std::vector<double>& sigma, std::vector<double>& resid) {
  cudaStream_t s = ctx->stream;
  const int m = A.m, n = A.n;
  double* av = pool.get<double>(m);
  double* atu = pool.get<double>(n);
  double* acc = pool.get<double>(8);
  Host h(ctx);
  sigma.assign(k, 0.0);
  resid.assign(k, 0.0);
  for (int i = 0; i < k; ++i) {
    double* v = Vd + (size_t)i * n;
    double* u = Ud + (size_t)i * m;
    zero(s, acc, 4);
    col_norms2_dense<double>(s, n, v, n, 1, acc);
    if (have_u) col_norms2_dense<double>(s, m, u, m, 1, acc + 1);
    CUCHK(cudaMemcpyAsync(h.at<double>(0), acc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    sync(s);
    const double nv = std::sqrt(*h.at<double>(0)), nu = have_u ? std::sqrt(*h.at<double>(8)) : 1.0;
    scal(s, n, 1.0 / nv, nullptr, v);
    if (have_u) scal(s, m, 1.0 / nu, nullptr, u);
    csr_spmm<double>(s, A.A64, 1, v, av);
    zero(s, acc, 4);
    if (have_u) {
      dot_accum(s, m, u, av, acc);
    } else {
      col_norms2_dense<double>(s, m, av, m, 1, acc);
    }
    CUCHK(cudaMemcpyAsync(h.at<double>(0), acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    sync(s);
    double sg = have_u ? *h.at<double>(0) : std::sqrt(*h.at<double>(0));
    if (!have_u) {
      CUCHK(cudaMemcpyAsync(u, av, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
      scal(s, m, sg > 0 ? 1.0 / sg : 0.0, nullptr, u);
    } else if (sg < 0) {
      scal(s, m, -1.0, nullptr, u);
      sg = -sg;
    }
    sigma[i] = sg;
    csr_spmm<double>(s, A.At64, 1, u, atu);
    axpby(s, m, -sg, u, 1.0, av);   // av = A v - s u
    axpby(s, n, -sg, v, 1.0, atu);  // atu = A^T u - s v
    zero(s, acc, 4);
    col_norms2_dense<double>(s, m, av, m, 1, acc);
    col_norms2_dense<double>(s, n, atu, n, 1, acc + 1);
    CUCHK(cudaMemcpyAsync(h.at<double>(0), acc, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    sync(s);
    resid[i] = std::sqrt(*h.at<double>(0) + *h.at<double>(8));
  }
}

// ---------------------------------------------------------------------------
// The whole method
// ---------------------------------------------------------------------------
// ||C|| estimated by L Lanczos steps on C (FP64, seeded random start, no
// reorthogonalisation: the extreme Ritz value needs none): the largest
// eigenvalue of the tridiagonal T_L, found by the one-CTA Jacobi solver.  A
// lower bound of ||C|| that converges quickly from below.  The host only
// gathers the scalars alpha_i, beta_i into T.
static double lanczos_normC(phsvds_ctx* ctx, Pool& pool, const COp<double>& op, int n, uint64_t seed, int L,
                            int64_t& mv) {
  cudaStream_t s = ctx->stream;
  Host h(ctx);
  L = std::max(1, std::min(L, std::min(n, LD)));
  double* v0 = pool.get<double>((size_t)n);
  double* v1 = pool.get<double>((size_t)n);
  double* w = pool.get<double>((size_t)n);
  double* d = pool.get<double>(2);
  double* T = pool.get<double>(LD * LD);
  double* S = pool.get<double>(LD * LD);
  double* th = pool.get<double>(LD);
  auto to_host = [&](const double* dv) {
    CUCHK(cudaMemcpyAsync(h.at<double>(0), dv, sizeof(double), cudaMemcpyDeviceToHost, s));
    sync(s);
    return *h.at<double>(0);
  };
  fill_random<double>(s, n, v1, seed, RS_NORM);
  zero(s, d, 1);
  col_norms2_dense<double>(s, n, v1, n, 1, d);
  const double n0 = std::sqrt(std::max(to_host(d), 0.0));
  if (!(n0 > 0)) return 0.0;
  scal(s, n, 1.0 / n0, nullptr, v1);
  zero(s, v0, (size_t)n);
  std::vector<double> al, be;
  double beta = 0.0;
  for (int i = 0; i < L; ++i) {
    op.apply(s, 1, v1, w);
    ++mv;
    zero(s, d, 1);
    dot_accum(s, n, v1, w, d);
    const double alpha = to_host(d);
    axpby(s, n, -alpha, v1, 1.0, w);
    if (i > 0) axpby(s, n, -beta, v0, 1.0, w);
    zero(s, d, 1);
    col_norms2_dense<double>(s, n, w, n, 1, d);
    const double b2 = to_host(d);
    if (!std::isfinite(alpha) || !std::isfinite(b2)) throw PhError{PHSVDS_ERR_NAN, "non-finite value in the norm estimate"};
    al.push_back(alpha);
    beta = std::sqrt(std::max(b2, 0.0));
    if (i + 1 == L || !(beta > 1e-14 * std::fabs(alpha))) break;
    be.push_back(beta);
    std::swap(v0, v1);
    CUCHK(cudaMemcpyAsync(v1, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    scal(s, n, 1.0 / beta, nullptr, v1);
  }
  const int jl = (int)al.size();
  double* hT = h.at<double>(1024);   // bytes [1024, 1024 + 8 LD^2)
  for (int c = 0; c < jl; ++c)
    for (int r = 0; r < jl; ++r)
      hT[r + c * jl] = r == c ? al[c] : (r == c + 1 || c == r + 1) ? be[std::min(r, c)] : 0.0;
  CUCHK(cudaMemcpyAsync(T, hT, sizeof(double) * jl * jl, cudaMemcpyHostToDevice, s));
  set_identity(s, jl, S, jl);
  jacobi_eig(s, jl, T, S, th, 1e-15, 30, nullptr);
  CUCHK(cudaMemcpyAsync(h.at<double>(0), th, sizeof(double) * jl, cudaMemcpyDeviceToHost, s));
  sync(s);
  double mx = 0.0;
  for (int i = 0; i < jl; ++i) mx = std::max(mx, *h.at<double>(8 * i));
  return mx;
}

static void solve_impl(phsvds_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci,
                       const double* va, int on_dev, int k, phsvds_target target, double tol, phsvds_precond precond,
                       const phsvds_opts& o, double* sigma, double* U, double* V, double* resid, phsvds_stats* st) {
  using clk = std::chrono::steady_clock;
  const auto tstart = clk::now();
  cudaStream_t s = ctx->stream;
  const bool largest = target == PHSVDS_LARGEST;
  const bool mixed = o.precision == PHSVDS_MIXED;
  const int b = std::max(1, std::min(o.block_size, k));
  Pool pool(s, ctx->mempool);
  RedScope red(pool, s);
  DevA A;
  const int64_t launches0 = g_launch_count;
  const bool given = precond == PHSVDS_PREC_GIVEN;
  upload_matrix(ctx, pool, A, m, n, nnz, rp, ci, va, on_dev, mixed,
                precond == PHSVDS_PREC_JACOBI || precond == PHSVDS_PREC_LEARNED || o.stage2_precond, 8);
  // a preconditioner M ~ A given by the caller (diagonal): stage 1 applies
  // M^{-1} M^{-T} through the Olsen machinery with d = m^2 and no shift
  double *Mdev = nullptr, *M2dev = nullptr;
  if (given) {
    Mdev = pool.get<double>(A.n);
    M2dev = pool.get<double>(A.n);
    CUCHK(cudaMemcpyAsync(Mdev, o.precond_M, sizeof(double) * A.n, cudaMemcpyHostToDevice, s));
    square(s, A.n, Mdev, M2dev);
  }
  const int precond1 = given ? (int)PHSVDS_PREC_JACOBI : (int)precond;
  const double* diag1 = given ? M2dev : A.diagC;
  // learned correction: network weights (FP32 from BF16) and feature planes on the device
  LearnedDev ld;
  if (precond == PHSVDS_PREC_LEARNED) {
    void* pdev = pool.get<uint16_t>(3024);
    CUCHK(cudaMemcpyAsync(pdev, o.learned_params, sizeof(uint16_t) * 3024, cudaMemcpyHostToDevice, s));
    float* feat = pool.get<float>((size_t)3 * A.n);
    CUCHK(cudaMemcpyAsync(feat, o.learned_features, sizeof(float) * 3 * A.n, cudaMemcpyHostToDevice, s));
    ld.feat = feat;
    ld.nx = o.grid_nx;
    ld.ny = o.grid_ny;
    ld.wf = pool.get<float>(3024);
    ld.wt = pool.get<float>(3024);
    ld.xin = pool.get<float>((size_t)8 * 4 * A.n);
    ld.a1 = pool.get<float>((size_t)8 * 16 * A.n);
    ld.a2 = pool.get<float>((size_t)8 * 16 * A.n);
    ld.yout = pool.get<float>((size_t)8 * A.n);
    ld.nrm2 = pool.get<double>(8);
    ld.stall_window = o.stall_window;
    cnn_weights(s, pdev, ld.wf, ld.wt);
  }
  // SpMM schedule
  COp<double> op64{&A.A64, &A.At64, A.Z64, A.n, (int)o.spmm};
  COp<float> op32{&A.A32, &A.At32, A.Z32, A.n, (int)o.spmm};
  bool cached64 = false, cached32 = false;
  if (o.spmm == PHSVDS_SPMM_AUTO) {
    op64 = tuned_spmm<double>(ctx, pool, A.A64, A.At64, A.Z64, A.n, spmm_width(b), &cached64, o.deterministic);
    if (mixed)
      op32 = tuned_spmm<float>(ctx, pool, A.A32, A.At32, A.Z32, A.n, spmm_width(b), &cached32, o.deterministic);
  }
  const int sch64 = op64.schedule;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->spmm_schedule = sch64;
  }
  double work0[2][PROF_NALL];
  std::memcpy(work0, g_work, sizeof(work0));
  if (o.profile) g_prof.start(1 << 16);
  // ---- stage 1
  const auto t1a = clk::now();
  const double tol_in = TOL_MARGIN * tol;
  // ||A|| of the user requirement (opts.norm_A): the switch test and stage 2;
  // stage 1's delta_C keeps its running largest Ritz value (Algorithm 1)
  int64_t mv_norm = 0;
  double thC0 = 0.0;
  if (o.norm_A > 0)
    thC0 = o.norm_A * o.norm_A;
  else if (o.norm_A < 0)
    thC0 = lanczos_normC(ctx, pool, op64, A.n, o.seed, 30, mv_norm);
  Stage1<double> s1(ctx, pool, A.n, k, o, largest, tol_in, EPS64, precond1, diag1, op64);
  s1.shift_free = given;
  s1.lp = &ld;
  s1.rec_r = o.record_r;
  s1.rec_max = o.record_r ? o.record_max : 0;
  s1.rec_every = o.record_every;
  int64_t iters32 = 0, mv32 = 0, jac32[4] = {0, 0, 0, 0}, stag32 = 0;
  std::unique_ptr<InnerSolver> jd;
  int64_t jd32_steps = 0, jd32_solves = 0;   // the FP32 stage's inner solves (mixed_inner = 2)
  double theta_max32 = 0.0;
  // on a stage-1 error the counters so far still reach the caller
  auto partial_stats = [&](const Stage1Out& a, const Stage1Out* b32) {
    if (!st) return;
    st->iters_stage1 = a.iters + (b32 ? b32->iters : 0);
    st->iters_stage1_fp32 = b32 ? b32->iters : 0;
    st->restarts = a.restarts + (b32 ? b32->restarts : 0);
    st->matvecs_A = st->matvecs_At = a.mv + (b32 ? b32->mv : 0);
    st->recorded = a.recorded;
    st->fell_back = a.fell_back | (b32 ? b32->fell_back : 0);
    st->fell_back_at = b32 && b32->fell_back ? b32->fell_back_at : a.fell_back_at;
    st->norm_A_est = std::sqrt(std::max(a.theta_max, b32 ? b32->theta_max : 0.0));
    st->kernel_launches = g_launch_count - launches0;
    st->t_stage1_ms = std::chrono::duration<double, std::milli>(clk::now() - t1a).count();
    st->t_total_ms = std::chrono::duration<double, std::milli>(clk::now() - tstart).count();
  };
  // optional initial guess (opts.init_V): host n x init_nv, column-major
  const int nx0 = o.init_V ? std::min(o.init_nv > 0 ? o.init_nv : k, A.n) : 0;
  double* X0d = nullptr;
  if (nx0) {
    X0d = pool.get<double>((size_t)A.n * nx0);
    CUCHK(cudaMemcpyAsync(X0d, o.init_V, sizeof(double) * A.n * nx0, cudaMemcpyHostToDevice, s));
  }
  if (mixed) {
    Stage1<float> s1f(ctx, pool, A.n, k, o, largest, tol_in, EPS32, precond1, diag1, op32);
    std::unique_ptr<InnerSolver> jdf;
    if (o.mixed_inner == 2 && (precond1 == PHSVDS_PREC_NONE || precond1 == PHSVDS_PREC_JACOBI)) {
      jdf = std::make_unique<InnerJD<float>>(ctx, pool, A.n, k, op32, o.inner_maxit, o.inner_tol, !o.profile);
      s1f.jd = jdf.get();
    }
    s1f.lp = &ld;
    s1f.shift_free = given;
    float* X0f = nullptr;
    if (nx0) {
      X0f = pool.get<float>((size_t)A.n * nx0);
      convert_f64_to_f32(s, (int64_t)A.n * nx0, X0d, X0f);
    }
    try {
      s1f.run(X0f, nx0);
    } catch (const PhError&) {
      partial_stats(s1.out, &s1f.out);
      throw;
    }
    if (s1f.out.fell_back) {
      s1.precond = s1f.precond;  // the FP64 continuation keeps the fallback
      s1.out.fell_back = 1;
      s1.out.fell_back_at = s1f.out.fell_back_at;
    }
    iters32 = s1f.out.iters;
    mv32 = s1f.out.mv;
    if (jdf) jd32_steps = jdf->steps, jd32_solves = jdf->solves;
    jac32[0] = s1f.out.jac_sweeps;
    jac32[1] = s1f.out.jac_rot;
    jac32[2] = s1f.out.jac_calls;
    jac32[3] = s1f.out.jac_dim;
    theta_max32 = s1f.out.theta_max;
    stag32 = s1f.out.stag_locks;
    // continue in FP64 from the FP32 eigenvectors (promoted)
    double* X0 = pool.get<double>((size_t)A.n * k);
    convert_f32_to_f64(s, (int64_t)A.n * k, s1f.Xl, X0);
    s1.out.restarts = s1f.out.restarts;
    s1.out.theta_max = s1f.out.theta_max;  // the ||C|| estimate carries over
    if (o.mixed_inner >= 1 && (s1.precond == PHSVDS_PREC_NONE || s1.precond == PHSVDS_PREC_JACOBI)) {
      jd = std::make_unique<InnerJD<float>>(ctx, pool, A.n, k, op32, o.inner_maxit, o.inner_tol, !o.profile);
      s1.jd = jd.get();
    }
    try {
      s1.run(X0, k);
    } catch (const PhError&) {
      Stage1Out f = s1f.out;
      f.restarts = 0;  // already carried into s1
      partial_stats(s1.out, &f);
      throw;
    }
  } else {
    if (o.stage1_inner == 1) {
      jd = std::make_unique<InnerJD<double>>(ctx, pool, A.n, k, op64, o.inner_maxit, o.inner_tol, !o.profile);
      s1.jd = jd.get();
    }
    try {
      s1.run(X0d, nx0);
    } catch (const PhError&) {
      partial_stats(s1.out, nullptr);
      throw;
    }
  }
  sync(s);
  const auto t1b = clk::now();
  double normA = std::sqrt(std::max(std::max(s1.out.theta_max, theta_max32), thC0));
  // stage-1 triplets u = A v / ||A v||
  double* Vd = pool.get<double>((size_t)A.n * k);
  double* Ud = pool.get<double>((size_t)A.m * k);
  CUCHK(cudaMemcpyAsync(Vd, s1.Xl, sizeof(double) * A.n * k, cudaMemcpyDeviceToDevice, s));
  std::vector<double> sg, rs;
  final_triplets(ctx, pool, A, k, Vd, Ud, false, sg, rs);
  int64_t mvA = s1.out.mv + mv32 + k + mv_norm, mvAt = s1.out.mv + mv32 + k + mv_norm;
  bool need2 = false;
  const double floor = o.eps_factor * EPS64;
  for (int i = 0; i < k; ++i)
    if (tol < floor * normA / std::max(sg[i], 1e-300) || !(rs[i] < tol_in * normA)) need2 = true;
  int64_t it2 = 0, rs2 = 0, inner2_steps = 0, inner2_solves = 0;
  double t2ms = 0.0;
  if (need2 && o.stage2) {
    const auto t2a = clk::now();
    std::vector<double> lam = s1.out.lam;
    double* Xv = s1.Xl;
    F64Ctx f(ctx, pool, A);
    if (o.rayleigh_ritz) {
      // basis for the post-process: locked vectors + best remaining Ritz vectors
      const int extra = std::max(0, std::min(o.min_restart - k, s1.j - (int)s1.final_conv.size()));
      double* Ext = pool.get<double>((size_t)A.n * std::max(extra, 1));
      if (extra > 0) {
        Host h(ctx);
        int* hi = h.at<int>(0);
        int ne = 0;
        for (int i = 0; i < s1.j && ne < extra; ++i) {
          const bool c = std::find(s1.final_conv.begin(), s1.final_conv.end(), i) != s1.final_conv.end();
          if (!c) hi[ne++] = s1.final_ord[i];
        }
        int* didx = pool.get<int>(LD);
        CUCHK(cudaMemcpyAsync(didx, hi, sizeof(int) * ne, cudaMemcpyHostToDevice, s));
        gather_cols(s, s1.j, s1.S, LD, didx, ne, s1.Scols, LD, nullptr, nullptr);
        tall_times_small<double>(s, A.n, s1.V, A.n, s1.j, s1.Scols, LD, ne, Ext, A.n, nullptr, 0, nullptr, nullptr);
      }
      double* Xrr = pool.get<double>((size_t)A.n * k);
      int64_t mvrr = 0;
      lam = rayleigh_ritz_post(ctx, pool, A, op64, s1.Xl, k, Ext, extra, largest, o.seed, Xrr, mvrr);
      mvA += mvrr;
      mvAt += mvrr;
      Xv = Xrr;
    }
    std::vector<double> sig_s(k);
    for (int i = 0; i < k; ++i) sig_s[i] = std::sqrt(std::max(lam[i], 0.0));
    std::unique_ptr<InnerJD2> jd2;
    if (o.stage2_inner == 1) {
      // the targets stage 1 resolved go first and the tiny ones (sigma~ <=
      // sqrt(eps) ||A||, whose u~ is random) last, each group in its order,
      // so that accurate guesses lock before the ambiguous shifts near zero
      std::vector<int> ord2;
      for (int pass = 0; pass < 2; ++pass)
        for (int i = 0; i < k; ++i)
          if ((sig_s[i] <= std::sqrt(EPS64) * normA) == (pass == 1)) ord2.push_back(i);
      bool moved = false;
      for (int i = 0; i < k; ++i) moved = moved || ord2[i] != i;
      if (moved) {
        double* Xo = pool.get<double>((size_t)A.n * k);
        std::vector<double> so(k);
        for (int i = 0; i < k; ++i) {
          so[i] = sig_s[ord2[i]];
          CUCHK(cudaMemcpyAsync(Xo + (size_t)i * A.n, Xv + (size_t)ord2[i] * A.n, sizeof(double) * A.n,
                                cudaMemcpyDeviceToDevice, s));
        }
        sig_s = so;
        Xv = Xo;
      }
      jd2 = std::make_unique<InnerJD2>(ctx, pool, f, o.inner2_maxit, o.inner2_patience, !o.profile);
    }
    Stage2 s2(ctx, pool, f, A, k, o, tol_in, normA);
    s2.jd2 = jd2.get();
    if (given)
      s2.set_precond(2, Mdev, 0.0);
    else if (o.stage2_precond && !largest)
      s2.set_precond(1, A.diagC, EPS64 * normA * normA);
    s2.run(sig_s, Xv);
    mvA += s2.mv;
    mvAt += s2.mv;
    it2 = s2.iters;
    rs2 = s2.restarts;
    if (jd2) inner2_steps = jd2->steps, inner2_solves = jd2->solves;
    // split x = [v; u]
    for (int i = 0; i < k; ++i) {
      CUCHK(cudaMemcpyAsync(Vd + (size_t)i * A.n, s2.Xl + (size_t)i * s2.N, sizeof(double) * A.n,
                            cudaMemcpyDeviceToDevice, s));
      CUCHK(cudaMemcpyAsync(Ud + (size_t)i * A.m, s2.Xl + (size_t)i * s2.N + A.n, sizeof(double) * A.m,
                            cudaMemcpyDeviceToDevice, s));
    }
    final_triplets(ctx, pool, A, k, Vd, Ud, true, sg, rs);
    mvA += 2 * k;
    mvAt += k;
    sync(s);
    t2ms = std::chrono::duration<double, std::milli>(clk::now() - t2a).count();
  }
  // order: ascending (smallest) / descending (largest)
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b2) { return largest ? sg[a] > sg[b2] : sg[a] < sg[b2]; });
  Host h(ctx);
  for (int i = 0; i < k; ++i) {
    const int src = ord[i];
    sigma[i] = sg[src];
    if (resid) resid[i] = rs[src];
    if (V) CUCHK(cudaMemcpyAsync(V + (size_t)i * A.n, Vd + (size_t)src * A.n, sizeof(double) * A.n,
                                 cudaMemcpyDeviceToHost, s));
    if (U) CUCHK(cudaMemcpyAsync(U + (size_t)i * A.m, Ud + (size_t)src * A.m, sizeof(double) * A.m,
                                 cudaMemcpyDeviceToHost, s));
  }
  sync(s);
  double cls_ms[PROF_NALL] = {};
  int64_t cls_n[PROF_NALL] = {};
  if (o.profile) g_prof.finish(cls_ms, cls_n);
  if (st) {
    for (int c = 0; c < PROF_NALL; ++c) {
      st->t_class_ms[c] = cls_ms[c];
      st->n_class[c] = cls_n[c];
    }
    st->kernel_launches = g_launch_count - launches0;
    const int64_t nc_c = cls_n[PROF_CSPMM] + cls_n[PROF_CSPMM + PROF_F32];
    st->spmm_c_calls = nc_c ? nc_c : (s1.out.mv + mv32) / std::max(1, spmm_width(b));
    st->spmm_c_ms = cls_ms[PROF_CSPMM] + cls_ms[PROF_CSPMM + PROF_F32];
    st->spmm_c_width = spmm_width(b);
    st->jacobi_sweeps = s1.out.jac_sweeps + jac32[0];
    st->jacobi_rotations = s1.out.jac_rot + jac32[1];
    st->jacobi_calls = s1.out.jac_calls + jac32[2];
    st->jacobi_dim_sum = s1.out.jac_dim + jac32[3];
    st->matvecs_A = mvA;
    st->matvecs_At = mvAt;
    st->iters_stage1 = s1.out.iters + iters32;
    st->iters_stage1_fp32 = iters32;
    st->iters_stage2 = it2;
    st->restarts = s1.out.restarts + rs2;
    st->switched = need2 && o.stage2;
    st->norm_A_est = normA;
    st->fell_back = s1.out.fell_back;
    st->fell_back_at = s1.out.fell_back_at;
    st->recorded = s1.out.recorded;
    st->stage1_stagnation_locks = s1.out.stag_locks + stag32;
    st->inner_steps = (jd ? jd->steps : 0) + jd32_steps;
    st->inner_solves = (jd ? jd->solves : 0) + jd32_solves;
    st->inner2_steps = inner2_steps;
    st->inner2_solves = inner2_solves;
    st->t_stage1_ms = std::chrono::duration<double, std::milli>(t1b - t1a).count();
    st->t_stage2_ms = t2ms;
    st->t_total_ms = std::chrono::duration<double, std::milli>(clk::now() - tstart).count();
    st->spmm_schedule = sch64;
    st->spmm_plan_cached = (o.spmm == PHSVDS_SPMM_AUTO) && cached64 && (!mixed || cached32);
    st->spmm_schedule_f32 = mixed ? op32.schedule : 0;
    for (int c = 0; c < PROF_NALL; ++c) {
      st->class_flops[c] = g_work[0][c] - work0[0][c];
      st->class_bytes[c] = g_work[1][c] - work0[1][c];
    }
  }
  (void)iters32;
}

// ---------------------------------------------------------------------------
// Algorithm 3 (Sec. 4): dynamic switching between GD+k on C and on B under
// preconditioning, for the k smallest triplets
// ---------------------------------------------------------------------------
// Runs alternate between GD+k on C (the stage-1 operator with the shift-free
// preconditioner of its family) and GD+k on B (targets: the positive
// eigenvalues nearest zero, with the B preconditioner of the same family),
// each starting from the other's approximations ([v; A v / ||A v||] / sqrt 2
// into B, the normalised v-part out of it); a run's rate is the mean slope of
// log ||r|| of its first unconverged target.  The loop follows the
// algorithm's steps (initial tests on C then B; the faster approach runs
// again with maxIter doubled when it repeats and halved when it switches; a
// run that locks a pair ends the deciding), and its end the four final
// branches: all found on B; all found on C (the two-stage method from those
// vectors); C faster (the two-stage method from C's current vectors); B
// faster (B to the end).  The two-stage endings are the ordinary solve with
// the current vectors as its initial guess (opts.init_V).
static double convergence_rate(const std::vector<double>& hist) {
  std::vector<double> h;
  for (double x : hist)
    if (x > 0) h.push_back(x);
  if (h.size() < 2) return 0.0;
  return (std::log(h.back()) - std::log(h.front())) / (double)(h.size() - 1);
}

static void dynamic_impl(phsvds_ctx* ctx, int64_t m, int64_t n, int64_t nnz, const int64_t* rp, const int32_t* ci,
                         const double* va, int on_dev, int k, double tol, phsvds_precond precond,
                         const phsvds_opts& o, double* sigma, double* U, double* V, double* resid, phsvds_stats* st) {
  using clk = std::chrono::steady_clock;
  const auto tstart = clk::now();
  cudaStream_t s = ctx->stream;
  Pool pool(s, ctx->mempool);
  RedScope red(pool, s);
  DevA A;
  const int64_t launches0 = g_launch_count;
  const bool given = precond == PHSVDS_PREC_GIVEN, jac = precond == PHSVDS_PREC_JACOBI;
  upload_matrix(ctx, pool, A, m, n, nnz, rp, ci, va, on_dev, false, jac, 8);
  const int N = A.m + A.n;
  const double tol_in = TOL_MARGIN * tol;
  // the shift-free preconditioners of Sec. 4 in the Olsen form
  double *Mdev = nullptr, *dC = nullptr;
  BPrecond bpre;
  if (given) {
    Mdev = pool.get<double>(A.n);
    dC = pool.get<double>(A.n);
    CUCHK(cudaMemcpyAsync(Mdev, o.precond_M, sizeof(double) * A.n, cudaMemcpyHostToDevice, s));
    square(s, A.n, Mdev, dC);                 // C: M^{-1} M^{-T} = diag(1 / m_j^2)
    bpre.init(s, pool, A, 2, Mdev, 0.0);      // B: [0 M^{-1}; M^{-T} 0]
  } else if (jac) {
    dC = A.diagC;                              // C: diag(C)^{-1}
    Host h(ctx);
    // guard of the B form: eps * max diag(C)
    double* gmax = pool.get<double>(1);
    zero(s, gmax, 1);
    col_norms2_dense<double>(s, A.n, A.diagC, A.n, 1, gmax);   // ||diag(C)||^2 >= max^2
    CUCHK(cudaMemcpyAsync(h.at<double>(0), gmax, sizeof(double), cudaMemcpyDeviceToHost, s));
    sync(s);
    bpre.init(s, pool, A, 1, A.diagC, EPS64 * std::sqrt(*h.at<double>(0)));
  }
  const int prec1 = (given || jac) ? (int)PHSVDS_PREC_JACOBI : (int)PHSVDS_PREC_NONE;
  const int b = std::max(1, std::min(o.block_size, k));
  bool cached = false;
  COp<double> opC = tuned_spmm<double>(ctx, pool, A.A64, A.At64, A.Z64, A.n, spmm_width(b), &cached,
                                       o.deterministic);
  BOp opB{&A.A64, &A.At64, A.m, A.n};
  double* curX = pool.get<double>((size_t)A.n * k);
  double* X0B = pool.get<double>((size_t)N * k);
  double* nrm = pool.get<double>(2);
  bool have_x = false;
  double normA = 0.0;
  int64_t iters_total = 0, mv_total = 0;
  struct Run {
    bool done = false;
    int nconv = 0;
    double rate = 0.0;
    int64_t iters = 0;
  };
  double* Xfin = nullptr;   // B's final vectors (N x k) for the B endings
  auto runC = [&](int64_t iters) {
    Stage1<double> sC(ctx, pool, A.n, k, o, false, tol_in, EPS64, prec1, dC, opC);
    sC.shift_free = true;
    sC.stop_after = iters;
    sC.run(have_x ? curX : nullptr, have_x ? k : 0);
    sync(s);
    Run r;
    r.done = !sC.partial;
    r.nconv = r.done ? k : sC.nlock;
    r.rate = convergence_rate(sC.history);
    r.iters = sC.out.iters;
    CUCHK(cudaMemcpyAsync(curX, r.done ? sC.Xl : sC.Xpart, sizeof(double) * A.n * k, cudaMemcpyDeviceToDevice, s));
    have_x = true;
    normA = std::max(normA, std::sqrt(std::max(sC.out.theta_max, 0.0)));
    iters_total += sC.out.iters;
    mv_total += sC.out.mv;
    return r;
  };
  auto runB = [&](int64_t iters) {
    Host h(ctx);
    if (have_x) {  // [v; A v / ||A v||] / sqrt(2)
      for (int c = 0; c < k; ++c) {
        double* xc = X0B + (size_t)c * N;
        const double* vc = curX + (size_t)c * A.n;
        CUCHK(cudaMemcpyAsync(xc, vc, sizeof(double) * A.n, cudaMemcpyDeviceToDevice, s));
        csr_spmm<double>(s, A.A64, 1, vc, xc + A.n);
        zero(s, nrm, 2);
        col_norms2_dense<double>(s, A.n, xc, A.n, 1, nrm);
        col_norms2_dense<double>(s, A.m, xc + A.n, A.m, 1, nrm + 1);
        CUCHK(cudaMemcpyAsync(h.at<double>(0), nrm, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        sync(s);
        const double nv = std::sqrt(*h.at<double>(0)), nu = std::sqrt(*h.at<double>(8));
        scal(s, A.n, nv > 0 ? 1.0 / (nv * std::sqrt(2.0)) : 0.0, nullptr, xc);
        scal(s, A.m, nu > 0 ? 1.0 / (nu * std::sqrt(2.0)) : 0.0, nullptr, xc + A.n);
      }
    }
    Stage1<double, BOp> sB(ctx, pool, N, k, o, false, tol_in, EPS64, PHSVDS_PREC_NONE, nullptr, opB);
    sB.bmode = true;
    sB.bp = bpre.mode ? &bpre : nullptr;
    sB.stop_after = iters;
    sB.run(have_x ? X0B : nullptr, have_x ? k : 0);
    sync(s);
    Run r;
    r.done = !sB.partial;
    r.nconv = r.done ? k : sB.nlock;
    r.rate = convergence_rate(sB.history);
    r.iters = sB.out.iters;
    const double* X = r.done ? sB.Xl : sB.Xpart;
    if (r.done) {
      if (!Xfin) Xfin = pool.get<double>((size_t)N * k);
      CUCHK(cudaMemcpyAsync(Xfin, X, sizeof(double) * N * k, cudaMemcpyDeviceToDevice, s));
    }
    for (int c = 0; c < k; ++c) {  // the normalised v-parts
      CUCHK(cudaMemcpyAsync(curX + (size_t)c * A.n, X + (size_t)c * N, sizeof(double) * A.n,
                            cudaMemcpyDeviceToDevice, s));
      zero(s, nrm, 1);
      col_norms2_dense<double>(s, A.n, curX + (size_t)c * A.n, A.n, 1, nrm);
      CUCHK(cudaMemcpyAsync(h.at<double>(0), nrm, sizeof(double), cudaMemcpyDeviceToHost, s));
      sync(s);
      const double nv = std::sqrt(*h.at<double>(0));
      scal(s, A.n, nv > 0 ? 1.0 / nv : 0.0, nullptr, curX + (size_t)c * A.n);
    }
    have_x = true;
    normA = std::max(normA, sB.out.theta_max);
    iters_total += sB.out.iters;
    mv_total += sB.out.mv;
    return r;
  };
  const int init_iter = o.dyn_init_iter;
  int runs = 0, switches = 0, jexp = 0;
  int64_t max_iter = init_iter;
  Run last_C = runC(init_iter), last_B = runB(init_iter);
  runs = 2;
  int num_conv = std::max(last_C.nconv, last_B.nconv);
  char prev = 'B';
  bool undecided = true;
  while (switches < o.dyn_max_switch && undecided) {
    const char choice = last_C.rate < last_B.rate ? 'C' : 'B';
    if ((switches == 0 && num_conv > 0) || num_conv > 1) {
      undecided = false;
    } else {
      jexp = choice == prev ? jexp + 1 : jexp / 2;   // Algorithm 3: double on a repeat, halve on a switch
      max_iter = (int64_t)init_iter << jexp;
    }
    ++switches;
    Run r = choice == 'C' ? runC(max_iter) : runB(max_iter);
    ++runs;
    (choice == 'C' ? last_C : last_B) = r;
    num_conv = r.nconv;
    prev = choice;
    if (r.done) break;
  }
  const char faster = last_C.rate < last_B.rate ? 'C' : 'B';
  const bool prev_done = prev == 'C' ? last_C.done : last_B.done;
  int route;
  if (prev_done && prev == 'B') {
    route = 3;                                  // all found on B
  } else if (prev_done && prev == 'C') {
    route = 1;                                  // all found on C: the two-stage method from them
  } else if (faster == 'C') {
    route = 2;                                  // C faster: the two-stage method from C's vectors
  } else {
    route = 4;                                  // B faster: B to the end
    Run r = runB(0);
    ++runs;
    (void)r;
  }
  if (route == 1 || route == 2) {
    // the ordinary solve, warm-started from the current approximations
    Host h(ctx);
    std::vector<double> hx((size_t)A.n * k);
    CUCHK(cudaMemcpyAsync(hx.data(), curX, sizeof(double) * A.n * k, cudaMemcpyDeviceToHost, s));
    sync(s);
    phsvds_opts o2 = o;
    o2.dynamic = 0;
    o2.init_V = hx.data();
    o2.init_nv = k;
    phsvds_precond p2 = precond;
    solve_impl(ctx, m, n, nnz, rp, ci, va, on_dev, k, PHSVDS_SMALLEST, tol, p2, o2, sigma, U, V, resid, st);
    if (st) {
      st->iters_stage1 += iters_total;
      st->matvecs_A += mv_total;
      st->matvecs_At += mv_total;
      st->dynamic_route = route;
      st->dynamic_runs = runs;
      st->dynamic_switches = switches;
      st->t_total_ms = std::chrono::duration<double, std::milli>(clk::now() - tstart).count();
    }
    return;
  }
  // B endings: the triplets from the augmented vectors
  double* Vd = pool.get<double>((size_t)A.n * k);
  double* Ud = pool.get<double>((size_t)A.m * k);
  for (int c = 0; c < k; ++c) {
    CUCHK(cudaMemcpyAsync(Vd + (size_t)c * A.n, Xfin + (size_t)c * N, sizeof(double) * A.n,
                          cudaMemcpyDeviceToDevice, s));
    CUCHK(cudaMemcpyAsync(Ud + (size_t)c * A.m, Xfin + (size_t)c * N + A.n, sizeof(double) * A.m,
                          cudaMemcpyDeviceToDevice, s));
  }
  std::vector<double> sg, rs;
  final_triplets(ctx, pool, A, k, Vd, Ud, true, sg, rs);
  std::vector<int> ord(k);
  for (int i = 0; i < k; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a2, int b2) { return sg[a2] < sg[b2]; });
  for (int i = 0; i < k; ++i) {
    const int src = ord[i];
    sigma[i] = sg[src];
    if (resid) resid[i] = rs[src];
    if (V) CUCHK(cudaMemcpyAsync(V + (size_t)i * A.n, Vd + (size_t)src * A.n, sizeof(double) * A.n,
                                 cudaMemcpyDeviceToHost, s));
    if (U) CUCHK(cudaMemcpyAsync(U + (size_t)i * A.m, Ud + (size_t)src * A.m, sizeof(double) * A.m,
                                 cudaMemcpyDeviceToHost, s));
  }
  sync(s);
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->iters_stage1 = iters_total;
    st->matvecs_A = st->matvecs_At = mv_total + 2 * k;
    st->norm_A_est = normA;
    st->dynamic_route = route;
    st->dynamic_runs = runs;
    st->dynamic_switches = switches;
    st->kernel_launches = g_launch_count - launches0;
    st->t_total_ms = std::chrono::duration<double, std::milli>(clk::now() - tstart).count();
  }
}

}  // namespace ph

// ===========================================================================
// C ABI
// ===========================================================================
using namespace ph;

static phsvds_status set_err(phsvds_ctx* c, phsvds_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

template <typename T>
static phsvds_status ata_api(phsvds_handle h, int schedule, int lanes_a, int lanes_at, int64_t m, int64_t n,
                             int64_t nnz, const int32_t* rp, const int32_t* ci, const T* va, const int32_t* cp,
                             const int32_t* ri, const T* cv, int b, const T* X, T* Y, T* z) {
  auto lanes_ok = [](int l) {
    const int a = l < 0 ? -l : l;
    return a == 0 || a == 1 || a == 2 || a == 4 || a == 8 || a == 16;
  };
  if (!h || m < 1 || n < 1 || m > INT32_MAX || n > INT32_MAX || nnz < 0 || nnz > INT32_MAX || !rp || !X || !Y ||
      (b != 1 && b != 2 && b != 4 && b != 8) || (schedule != 1 && schedule != 2) ||
      (schedule == 2 && (!cp || !z)) || (nnz > 0 && (!ci || !va)) ||
      (schedule == 2 && nnz > 0 && (!ri || !cv)) || !lanes_ok(lanes_a) || !lanes_ok(lanes_at))
    return set_err(h, PHSVDS_ERR_INVALID, "invalid SpMM arguments");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
  // nnz only picks the automatic lane width (mean row length)
  SparseView<T> A{(int)m, (int)n, nnz, rp, ci, va};
  SparseView<T> At{(int)n, (int)m, nnz, cp, ri, cv};
  if (schedule == 1)
    ata_fused<T>(h->stream, A, (int)n, b, X, Y, lanes_a);
  else
    ata_two_phase<T>(h->stream, A, At, b, X, Y, z, lanes_a, lanes_at);
  e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" {

phsvds_status phsvds_default_opts(phsvds_opts* o) {
  if (!o) return PHSVDS_ERR_INVALID;
  o->block_size = 1;
  o->max_basis = 35;
  o->min_restart = 21;
  o->max_restarts = 10000;
  o->eps_factor = 4.0;
  o->precision = PHSVDS_FP64;
  o->spmm = PHSVDS_SPMM_AUTO;
  o->stage2 = 1;
  o->rayleigh_ritz = 1;
  o->seed = 0;
  o->time_limit_s = 0.0;
  o->profile = 0;
  o->learned_params = nullptr;
  o->learned_features = nullptr;
  o->grid_nx = o->grid_ny = 0;
  o->stall_window = 200;
  o->record_r = nullptr;
  o->record_max = 0;
  o->record_every = 0;
  o->projected_solver = 2;
  o->init_V = nullptr;
  o->init_nv = 0;
  o->mixed_inner = 1;
  o->inner_maxit = 60;
  o->inner_tol = 1e-3;
  o->stage2_precond = 0;
  o->precond_M = nullptr;
  o->stage2_inner = 0;
  o->inner2_maxit = 300;
  o->inner2_patience = 25;
  o->dynamic = 0;
  o->dyn_init_iter = 50;
  o->dyn_max_switch = 8;
  o->deterministic = 1;
  o->norm_A = 0.0;
  o->stage1_inner = 0;
  return PHSVDS_OK;
}

phsvds_status phsvds_create(phsvds_handle* out, int device, void* stream) {
  if (!out) return PHSVDS_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PHSVDS_ERR_CUDA;
  if (cudaSetDevice(device) != cudaSuccess) return PHSVDS_ERR_CUDA;
  phsvds_ctx* c = new phsvds_ctx();
  c->device = device;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    // an ordinary stream: ordered with the legacy default stream, so work the
    // caller queued there (input preparation) completes before the library's
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault) != cudaSuccess) {
      delete c;
      return PHSVDS_ERR_CUDA;
    }
    c->own_stream = true;
  }
  c->host_bytes = 1 << 16;
  if (cudaMallocHost(&c->host, c->host_bytes) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return PHSVDS_ERR_OOM;
  }
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  if (cudaMemPoolCreate(&c->mempool, &props) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(c->mempool, cudaMemPoolAttrReleaseThreshold, &keep);
  } else {
    cudaGetLastError();
    c->mempool = nullptr;  // fall back to the device's default pool
  }
  *out = c;
  return PHSVDS_OK;
}

void phsvds_destroy(phsvds_handle h) {
  if (!h) return;
  cudaSetDevice(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->mempool) cudaMemPoolDestroy(h->mempool);
  if (h->host) cudaFreeHost(h->host);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

const char* phsvds_last_error(phsvds_handle h) { return h ? h->err.c_str() : "null handle"; }

const char* phsvds_status_string(phsvds_status s) {
  switch (s) {
    case PHSVDS_OK: return "ok";
    case PHSVDS_ERR_INVALID: return "invalid argument";
    case PHSVDS_ERR_NOT_CONVERGED: return "not converged";
    case PHSVDS_ERR_BREAKDOWN: return "breakdown";
    case PHSVDS_ERR_NAN: return "NaN or Inf";
    case PHSVDS_ERR_TIMEOUT: return "time limit";
    case PHSVDS_ERR_CUDA: return "CUDA error";
    case PHSVDS_ERR_OOM: return "out of device memory";
  }
  return "unknown";
}

phsvds_status phsvds_sync(phsvds_handle h) {
  if (!h) return PHSVDS_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

phsvds_status phsvds_solve(phsvds_handle h, int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                           const int32_t* col_idx, const double* val, int ptr_on_device, int k, phsvds_target target,
                           double tol, phsvds_precond precond, const phsvds_opts* opts, double* sigma, double* U,
                           double* V, double* resid, phsvds_stats* stats) {
  if (!h) return PHSVDS_ERR_INVALID;
  h->err.clear();
  phsvds_opts o;
  phsvds_default_opts(&o);
  if (opts) o = *opts;
  if (m < n || n < 1 || nnz < 0 || nnz >= (int64_t)1 << 31 || m >= (int64_t)1 << 31 || !row_ptr ||
      (nnz > 0 && (!col_idx || !val)) || !sigma)
    return set_err(h, PHSVDS_ERR_INVALID, "need m >= n >= 1, nnz < 2^31, non-null CSR arrays and sigma");
  if (k < 1 || k > n || k >= o.min_restart || k + o.max_basis > LD)
    return set_err(h, PHSVDS_ERR_INVALID, "need 1 <= k <= n, k < min_restart and k + max_basis <= 64");
  if (o.block_size < 1 || o.block_size > 8 || o.max_basis < 4 || o.max_basis + 8 > LD ||
      o.min_restart < 2 * std::min(o.block_size, k) ||
      o.max_basis - o.min_restart < std::min(o.block_size, k) || !(tol > 0) ||
      o.max_restarts < 1 || (target != PHSVDS_SMALLEST && target != PHSVDS_LARGEST) ||
      (precond != PHSVDS_PREC_NONE && precond != PHSVDS_PREC_JACOBI && precond != PHSVDS_PREC_LEARNED &&
       precond != PHSVDS_PREC_GIVEN) ||
      o.max_basis > n)
    return set_err(h, PHSVDS_ERR_INVALID,
                   "invalid options (block b in 1..8, 2b <= min_restart <= max_basis - b, max_basis <= min(n,56))");
  if (precond == PHSVDS_PREC_LEARNED &&
      (!o.learned_params || !o.learned_features || o.grid_nx < 1 || o.grid_ny < 1 ||
       (int64_t)o.grid_nx * o.grid_ny != n || o.stall_window < 0))
    return set_err(h, PHSVDS_ERR_INVALID, "learned correction needs params, features and grid_nx * grid_ny = n");
  if (o.record_r && (o.record_max < 0 || o.record_every < 1))
    return set_err(h, PHSVDS_ERR_INVALID, "recording needs record_max >= 0 and record_every >= 1");
  if (o.stage2_precond != 0 && o.stage2_precond != 1)
    return set_err(h, PHSVDS_ERR_INVALID, "stage2_precond must be 0 or 1");
  if ((o.stage1_inner != 0 && o.stage1_inner != 1) ||
      (o.stage1_inner == 1 && (o.precision != PHSVDS_FP64 || (precond != PHSVDS_PREC_NONE &&
                                                               precond != PHSVDS_PREC_JACOBI) || o.dynamic)))
    return set_err(h, PHSVDS_ERR_INVALID,
                   "stage1_inner must be 0 or 1 (1 with FP64, no or the Jacobi preconditioner, not dynamic)");
  if (!std::isfinite(o.norm_A) || (o.dynamic != 0 && o.norm_A != 0.0))
    return set_err(h, PHSVDS_ERR_INVALID, "norm_A must be finite (and 0 with dynamic = 1)");
  if (o.dynamic != 0 && (o.dynamic != 1 || target != PHSVDS_SMALLEST || o.dyn_init_iter < 1 ||
                         o.dyn_max_switch < 0 || o.precision != PHSVDS_FP64 || precond == PHSVDS_PREC_LEARNED ||
                         o.init_V))
    return set_err(h, PHSVDS_ERR_INVALID,
                   "dynamic = 1 needs SMALLEST, FP64, no learned correction or init_V, dyn_init_iter >= 1, "
                   "dyn_max_switch >= 0");
  if ((o.stage2_inner != 0 && o.stage2_inner != 1) || o.inner2_maxit < 1 || o.inner2_patience < 1 ||
      (o.stage2_inner == 1 && (o.stage2_precond || precond == PHSVDS_PREC_GIVEN)))
    return set_err(h, PHSVDS_ERR_INVALID,
                   "stage2_inner must be 0 or 1 (1 not with a stage-2 preconditioner), inner2_maxit and "
                   "inner2_patience >= 1");
  if (precond == PHSVDS_PREC_GIVEN) {
    if (!o.precond_M || m != n)
      return set_err(h, PHSVDS_ERR_INVALID, "a given preconditioner needs opts.precond_M and a square A");
    for (int64_t i = 0; i < n; ++i)
      if (!std::isfinite(o.precond_M[i]) || o.precond_M[i] == 0.0)
        return set_err(h, PHSVDS_ERR_INVALID, "precond_M must be finite and nonzero");
  }
  if (o.mixed_inner < 0 || o.mixed_inner > 2 || o.inner_maxit < 1 || !(o.inner_tol > 0) || o.inner_tol >= 1)
    return set_err(h, PHSVDS_ERR_INVALID, "mixed_inner must be 0, 1 or 2, inner_maxit >= 1, 0 < inner_tol < 1");
  if (o.init_V && (o.init_nv < 0 || o.init_nv > o.max_basis || (o.init_nv == 0 && k > o.max_basis)))
    return set_err(h, PHSVDS_ERR_INVALID, "init_V needs 0 <= init_nv <= max_basis (0 = k columns)");
  try {
    CUCHK(cudaSetDevice(h->device));
    if (o.dynamic)
      dynamic_impl(h, m, n, nnz, row_ptr, col_idx, val, ptr_on_device, k, tol, precond, o, sigma, U, V, resid,
                   stats);
    else
      solve_impl(h, m, n, nnz, row_ptr, col_idx, val, ptr_on_device, k, target, tol, precond, o, sigma, U, V,
                 resid, stats);
  } catch (const PhError& e) {
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    double ms[PROF_NALL] = {};
    int64_t cnt[PROF_NALL] = {};
    g_prof.finish(ms, cnt);
    return set_err(h, e.st, e.msg);
  }
  return PHSVDS_OK;
}

phsvds_status phsvds_csr_to_csc_f64(phsvds_handle h, int64_t m, int64_t n, int64_t nnz, const int32_t* row_ptr,
                                    const int32_t* col_idx, const double* val, int32_t* csc_ptr, int32_t* csc_row,
                                    double* csc_val) {
  if (!h || m < 0 || n < 1 || nnz < 0 || !row_ptr || !csc_ptr) return PHSVDS_ERR_INVALID;
  try {
    CUCHK(cudaSetDevice(h->device));
    int* work = nullptr;
    CUCHK(cudaMallocAsync(&work, sizeof(int) * n, h->stream));
    csr_to_csc<double>(h->stream, (int)m, (int)n, nnz, row_ptr, col_idx, val, csc_ptr, csc_row, csc_val, work);
    CUCHK(cudaFreeAsync(work, h->stream));
    CUCHK(cudaGetLastError());
  } catch (const PhError& e) {
    return set_err(h, e.st, e.msg);
  }
  return PHSVDS_OK;
}

phsvds_status phsvds_ata_spmm_f64(phsvds_handle h, int schedule, int lanes_a, int lanes_at, int64_t m, int64_t n,
                                  int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                  const int32_t* csc_ptr, const int32_t* csc_row, const double* csc_val, int b,
                                  const double* X, double* Y, double* z) {
  return ata_api<double>(h, schedule, lanes_a, lanes_at, m, n, nnz, row_ptr, col_idx, val, csc_ptr, csc_row, csc_val,
                         b, X, Y, z);
}

phsvds_status phsvds_ata_spmm_f32(phsvds_handle h, int schedule, int lanes_a, int lanes_at, int64_t m, int64_t n,
                                  int64_t nnz, const int32_t* row_ptr, const int32_t* col_idx, const float* val,
                                  const int32_t* csc_ptr, const int32_t* csc_row, const float* csc_val, int b,
                                  const float* X, float* Y, float* z) {
  return ata_api<float>(h, schedule, lanes_a, lanes_at, m, n, nnz, row_ptr, col_idx, val, csc_ptr, csc_row, csc_val,
                        b, X, Y, z);
}

phsvds_status phsvds_jacobi_eig_f64(phsvds_handle h, int j, double* H, double* S, double* theta, double tol,
                                    int max_sweeps, int* sweeps_out) {
  if (!h || j < 1 || j > LD || !H || !S || !theta) return PHSVDS_ERR_INVALID;
  jacobi_eig_fast_ld(h->stream, j, H, j, S, j, theta, tol, max_sweeps, sweeps_out, tol, 0, 0, 0.0, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

phsvds_status phsvds_jacobi_eig_cluster_f64(phsvds_handle h, int j, double* H, double* S, double* theta, double tol,
                                            int max_sweeps, int* sweeps_out) {
  if (!h || j < 1 || j > LD || !H || !S || !theta) return PHSVDS_ERR_INVALID;
  jacobi_eig_cluster_ld(h->stream, j, H, j, S, j, theta, tol, max_sweeps, sweeps_out, tol, 0, 0, 0.0, nullptr);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

phsvds_status phsvds_jacobi_svd_f64(phsvds_handle h, int j, double* G, double* S, double* sig, double tol,
                                    int max_sweeps, int* sweeps_out) {
  if (!h || j < 1 || j > LD || !G || !S || !sig) return PHSVDS_ERR_INVALID;
  jacobi_svd(h->stream, j, G, S, sig, tol, max_sweeps, sweeps_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

phsvds_status phsvds_refined_vector_f64(phsvds_handle h, int j, const double* R, int ldr, const double* x0,
                                        const double* H, int ldh, int maxit, double tau, double* s1,
                                        double* out, int* steps_out) {
  if (!h || j < 1 || j > LD || ldr < j || ldh < j || maxit < 1 || !(tau >= 0.0) || !R || !H || !s1 || !out)
    return PHSVDS_ERR_INVALID;
  refined_inverse(h->stream, j, R, ldr, x0, H, ldh, maxit, tau, s1, out, steps_out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"

// ===========================================================================
// Kernel-level entry points of the tall-skinny dense steps
// ===========================================================================
template <typename T>
static phsvds_status block_cgs_api(phsvds_handle h, int64_t n, const T* P1, int ld1, int p1, const T* P2, int ld2,
                                   int p2, T* Tb, int ldt, int q, const double* Gsub, double* Gout, double* Tout) {
  if (!h || n < 1 || n > INT32_MAX || p1 < 0 || p2 < 0 || p1 + p2 > 64 || q < 1 || q > 8 || !Tb || ldt < n ||
      (p1 > 0 && (!P1 || ld1 < n)) || (p2 > 0 && (!P2 || ld2 < n)) || ((Gsub || Gout) && p1 + p2 == 0))
    return set_err(h, PHSVDS_ERR_INVALID, "invalid block Gram-Schmidt arguments");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
  Basis<T> P{P1, ld1, p1, P2, ld2, p2};
  cgs_pass<T>(h->stream, (int)n, P, Tb, ldt, q, Gsub, Gout, Tout);
  e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

template <typename T>
static phsvds_status tall_small_api(phsvds_handle h, int64_t n, const T* P, int ldp, int p, const double* Y, int ldy,
                                    int r, T* Out, int ldo, const T* Xs, int ldx, const double* theta,
                                    double* norms2) {
  if (!h || n < 1 || n > INT32_MAX || p < 1 || p > 64 || r < 1 || r > 64 || !P || ldp < n || !Y || ldy < p ||
      !Out || ldo < n || (theta && (!Xs || ldx < n)) || (Out == P && r > p))
    return set_err(h, PHSVDS_ERR_INVALID, "invalid tall-times-small arguments");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
  tall_times_small<T>(h->stream, (int)n, P, ldp, p, Y, ldy, r, Out, ldo, theta ? Xs : nullptr, ldx, theta, norms2);
  e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

extern "C" {

phsvds_status phsvds_block_cgs_f64(phsvds_handle h, int64_t n, const double* P1, int ld1, int p1, const double* P2,
                                   int ld2, int p2, double* T, int ldt, int q, const double* Gsub, double* Gout,
                                   double* Tout) {
  return block_cgs_api<double>(h, n, P1, ld1, p1, P2, ld2, p2, T, ldt, q, Gsub, Gout, Tout);
}

phsvds_status phsvds_block_cgs_f32(phsvds_handle h, int64_t n, const float* P1, int ld1, int p1, const float* P2,
                                   int ld2, int p2, float* T, int ldt, int q, const double* Gsub, double* Gout,
                                   double* Tout) {
  return block_cgs_api<float>(h, n, P1, ld1, p1, P2, ld2, p2, T, ldt, q, Gsub, Gout, Tout);
}

phsvds_status phsvds_tall_small_f64(phsvds_handle h, int64_t n, const double* P, int ldp, int p, const double* Y,
                                    int ldy, int r, double* Out, int ldo, const double* Xs, int ldx,
                                    const double* theta, double* norms2) {
  return tall_small_api<double>(h, n, P, ldp, p, Y, ldy, r, Out, ldo, Xs, ldx, theta, norms2);
}

phsvds_status phsvds_tall_small_f32(phsvds_handle h, int64_t n, const float* P, int ldp, int p, const double* Y,
                                    int ldy, int r, float* Out, int ldo, const float* Xs, int ldx,
                                    const double* theta, double* norms2) {
  return tall_small_api<float>(h, n, P, ldp, p, Y, ldy, r, Out, ldo, Xs, ldx, theta, norms2);
}

}  // extern "C"

// ===========================================================================
// Allocation-free A^T (A X): the two-phase product with its intermediate
// Z = A X held in a fixed array of the library's own device memory.  The array
// is placed in device memory when the library's device code is loaded, so a
// call allocates nothing; its address is looked up once per device.
// ===========================================================================
static __device__ __align__(256) double g_static_z[PHSVDS_STATIC_Z_MAX];

namespace {
constexpr int kStaticZDevices = 64;
std::mutex g_static_z_mu;
double* g_static_z_addr[kStaticZDevices] = {};
}  // namespace

extern "C" phsvds_status phsvds_ata_spmm_static_f64(phsvds_handle h, int64_t m, int64_t n, int64_t nnz,
                                                    const int32_t* row_ptr, const int32_t* col_idx, const double* val,
                                                    const int32_t* csc_ptr, const int32_t* csc_row,
                                                    const double* csc_val, int b, const double* X, double* Y) {
  if (!h || m < 1 || n < 1 || n > INT32_MAX || nnz < 0 || nnz > INT32_MAX || !row_ptr || !csc_ptr || !X || !Y ||
      (nnz > 0 && (!col_idx || !val || !csc_row || !csc_val)) || (b != 1 && b != 2 && b != 4 && b != 8))
    return set_err(h, PHSVDS_ERR_INVALID, "invalid SpMM arguments");
  if (m * b > PHSVDS_STATIC_Z_MAX)
    return set_err(h, PHSVDS_ERR_INVALID,
                   "m * b = " + std::to_string(m * b) + " exceeds the fixed scratch of " +
                       std::to_string(PHSVDS_STATIC_Z_MAX) + " doubles; use phsvds_ata_spmm_f64 with a caller buffer");
  if (h->device < 0 || h->device >= kStaticZDevices)
    return set_err(h, PHSVDS_ERR_INVALID, "device ordinal out of range for the fixed scratch");
  cudaError_t e = cudaSetDevice(h->device);
  if (e != cudaSuccess) return set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
  double* z = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_z_mu);
    z = g_static_z_addr[h->device];
    if (!z) {
      // first call on this device (h->device is current): find the array
      e = cudaGetSymbolAddress(reinterpret_cast<void**>(&z), g_static_z);
      if (e != cudaSuccess || !z)
        return set_err(h, PHSVDS_ERR_CUDA,
                       std::string("cannot locate the fixed SpMM scratch: ") + cudaGetErrorString(e));
      g_static_z_addr[h->device] = z;
    }
  }
  // Z needs no clearing: the first phase writes all m x b entries before the
  // second phase reads any of them.
  SparseView<double> A{(int)m, (int)n, nnz, row_ptr, col_idx, val};
  SparseView<double> At{(int)n, (int)m, nnz, csc_ptr, csc_row, csc_val};
  ata_two_phase<double>(h->stream, A, At, b, X, Y, z);
  e = cudaGetLastError();
  return e == cudaSuccess ? PHSVDS_OK : set_err(h, PHSVDS_ERR_CUDA, cudaGetErrorString(e));
}

// ===========================================================================
// Inner solves for the training data of the learned correction: CG on the
// normal operator, up to 8 right-hand sides in lockstep.
// ===========================================================================
extern "C" phsvds_status phsvds_normal_cg(phsvds_handle h, int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                          const int32_t* col_idx, const double* val, int ptr_on_device, double shift,
                                          int count, const double* R, double* X, double rtol, int maxit, int* iters) {
  if (!h || m < 1 || n < 1 || m < n || nnz < 0 || !row_ptr || count < 1 || !R || !X || !(rtol > 0) || maxit < 1 ||
      !std::isfinite(shift))
    return set_err(h, PHSVDS_ERR_INVALID, "invalid CG arguments");
  phsvds_status result = PHSVDS_OK;
  try {
    CUCHK(cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    Pool pool(s, h->mempool);
    DevA A;
    upload_matrix(h, pool, A, m, n, nnz, row_ptr, col_idx, val, ptr_on_device, false, false, 8);
    COp<double> op{&A.A64, &A.At64, A.Z64, A.n, 2};
    const size_t nn = (size_t)n;
    double* cm = pool.get<double>(nn * 8);   // column-major staging
    double *Xb = pool.get<double>(nn * 8), *Rb = pool.get<double>(nn * 8), *Pb = pool.get<double>(nn * 8),
           *Qb = pool.get<double>(nn * 8);
    double* sc = pool.get<double>(32);       // rr | rrn | rr0 | pq
    int* ic = pool.get<int>(32);             // act | iters | bad
    Host hb(h);
    for (int c0 = 0; c0 < count; c0 += 8) {
      const int bw = std::min(8, count - c0);
      const int b = bw <= 1 ? 1 : bw <= 2 ? 2 : bw <= 4 ? 4 : 8;  // SpMM widths; extra columns stay zero
      zero(s, cm, nn * b);
      CUCHK(cudaMemcpyAsync(cm, R + (size_t)c0 * n, sizeof(double) * nn * bw, cudaMemcpyHostToDevice, s));
      cm_to_rm<double>(s, (int)n, cm, (int)n, b, Rb);
      CUCHK(cudaMemcpyAsync(Pb, Rb, sizeof(double) * nn * b, cudaMemcpyDeviceToDevice, s));
      zero(s, Xb, nn * b);
      zero(s, sc, 32);
      CUCHK(cudaMemsetAsync(ic, 0, sizeof(int) * 32, s));
      // rr0 = rr = ||r||^2 (through the update kernel with alpha = 0: act = 0)
      cg_update(s, (int)n, b, Pb, Pb, Xb, Rb, sc, sc + 24, ic, sc);
      CUCHK(cudaMemcpyAsync(sc + 16, sc, sizeof(double) * 8, cudaMemcpyDeviceToDevice, s));
      int* ha = hb.at<int>(0);
      for (int c = 0; c < 8; ++c) ha[c] = c < bw ? 1 : 0;
      CUCHK(cudaMemcpyAsync(ic, ha, sizeof(int) * 8, cudaMemcpyHostToDevice, s));
      sync(s);
      const double tol2 = rtol * rtol;
      int it = 0;
      while (it < maxit) {
        op.apply(s, b, Pb, Qb);
        cg_pq(s, (int)n, b, shift, Pb, Qb, sc + 24);
        cg_update(s, (int)n, b, Pb, Qb, Xb, Rb, sc, sc + 24, ic, sc + 8);
        cg_dir(s, (int)n, b, Rb, Pb, sc, sc + 8, ic);
        cg_next(s, b, sc, sc + 8, sc + 16, tol2, sc + 24, ic, ic + 8, ic + 16);
        ++it;
        if (it % 10 == 0 || it == maxit) {
          CUCHK(cudaMemcpyAsync(ha, ic, sizeof(int) * 24, cudaMemcpyDeviceToHost, s));
          sync(s);
          if (ha[16]) throw PhError{PHSVDS_ERR_INVALID, "CG: A^T A - shift I is not positive definite"};
          bool any = false;
          for (int c = 0; c < b; ++c) any = any || ha[c];
          if (!any) break;
        }
      }
      CUCHK(cudaMemcpyAsync(ha, ic, sizeof(int) * 24, cudaMemcpyDeviceToHost, s));
      rm_to_cm<double>(s, (int)n, Xb, b, cm, (int)n);
      CUCHK(cudaMemcpyAsync(X + (size_t)c0 * n, cm, sizeof(double) * nn * bw, cudaMemcpyDeviceToHost, s));
      sync(s);
      for (int c = 0; c < bw; ++c) {
        if (iters) iters[c0 + c] = ha[8 + c];
        if (ha[c]) result = PHSVDS_ERR_NOT_CONVERGED;
      }
    }
  } catch (const PhError& e) {
    cudaStreamSynchronize(h->stream);
    cudaGetLastError();
    return set_err(h, e.st, e.msg);
  }
  if (result != PHSVDS_OK) set_err(h, result, "CG: maxit reached before rtol");
  return result;
}
