// Host orchestrator and C ABI (include/rqrcp.h).
//
// Every public call validates its arguments, takes its scratch from the
// handle and enqueues kernels on the handle's stream; nothing waits for the
// device inside a call, the pivot list never travels to the host, and the
// launch sequence depends only on (m, n, k, b, p), so a whole factorization
// can be captured in a CUDA graph once its scratch is reserved.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kernels.cuh"

struct rqrcp_handle_s {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 1;       // SMs the handle's launches may use (RQRCP_OPT_MAX_SMS)
  int dev_sms = 1;       // SMs of the device
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int* state = nullptr;  // [0] status word, [1] re-sample flag; barrier at byte 64,
                         // then the panel's group arrival counters (up to 40)
  std::string err;
  // instrumentation
  bool prof = false;
  std::vector<cudaEvent_t> events;  // pool, pairs (2i, 2i+1)
  std::vector<int> ev_phase;
  size_t ev_used = 0;
  double flops[RQRCP_NPHASE] = {};
  int64_t launches[RQRCP_NPHASE] = {};
  int64_t launch_total = 0;
  int cur_phase = 7;
  int fp64_emulation = 0;  // RQRCP_OPT_FP64_EMULATION
  int resample = 0;        // RQRCP_OPT_RESAMPLE: Alg. 5 instead of Eq. (3)
  int test_timeout = 0;    // RQRCP_OPT_TEST_BARRIER_TIMEOUT (rqrcp_sample_qrcp only)
  // persistent batched kernel (trqrcp_batched and the serving ring): teams of
  // bt_G CTAs, each with bt_team_bytes of scratch sized for bt_lim
  int bt_G = 16;                    // RQRCP_OPT_BATCH_TEAM
  rq::BatchLimits bt_lim{};
  rq::BatchLayout bt_L{};
  size_t bt_team_bytes = 0;
  int bt_teams = 0;                 // teams the scratch holds
  char* bt_scratch = nullptr;
  char* bt_ctl = nullptr;           // claim counter, exit counter, one barrier per team
  rqrcp_problem* bt_table = nullptr;  // device descriptor table
  rqrcp_problem* bt_stage = nullptr;  // page-locked staging of the table
  int bt_cap = 0;
  // serving ring (page-locked, mapped) and its device address
  char* ring_host = nullptr;
  rq::RequestRing* ring_dev = nullptr;
  int ring_cap = 0;
  int64_t ring_tail = 0;            // requests published by the host
  bool ring_running = false;
  bool bt_trace_clear = true;       // the batched phase timers restart at the next launch
  int bt_server_teams = 0;          // teams of the serving launch
  cudaEvent_t bt_copy_ev = nullptr; // completion of the last table copy from the staging
  bool bt_copy_pending = false;
  // rqrcp_factor_host: copy stream, its events, device pivots and tau
  cudaStream_t io_st = nullptr;
  std::vector<cudaEvent_t> io_ev;
  int64_t* io_jpvt = nullptr;
  double* io_tau = nullptr;
  int64_t io_cap = 0;
};

namespace {

using rq::GemmArgs;

constexpr int kMaxB = 128;
constexpr int kMaxEll = 192;
constexpr uint32_t kOmegaStream = 1;
constexpr uint32_t kResampleStreamBase = 0x100;

size_t align_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout of one call; a sizing pass runs with base == nullptr.
struct Work {
  double* omega = nullptr;    // l x m (also the re-sample matrix)
  double* B = nullptr;        // l x n sample
  int64_t* swaps = nullptr;   // b
  int64_t* map = nullptr;     // 1 + 10 b
  double* permbuf = nullptr;  // rows x 2b (column moves)
  double* cand = nullptr;     // 2 x sms x 4
  double* candcol = nullptr;  // 2 x sms x l
  double* ppart = nullptr;    // panel partial sums
  double* rowj = nullptr;     // 2 b
  double* T = nullptr;        // b x b
  double* Z = nullptr;        // b x n
  double* W = nullptr;        // b x n
  double* skpart = nullptr;   // split-K partial sums
  size_t skcap = 0;
  double* W11 = nullptr;      // b x b
  // TRQRCP / TUXV
  double* Wt = nullptr;       // k x n
  double* Ahat = nullptr;     // m x b
  double* YY = nullptr;       // b x k
  double* OY = nullptr;       // l x k
  // TUXV
  double* Yk = nullptr;       // m x k
  double* Rk = nullptr;       // k x n
  int64_t* jpvt = nullptr;    // n
  double* tau = nullptr;      // k
  double* tau2 = nullptr;     // k
  double* Tall = nullptr;     // ceil(k/b) x b x b
  double* F = nullptr;        // max(m, n) x k copy of reflectors
  double* svd = nullptr;      // 5 k x k + k: X, G, Vx, Ux, Vs and raw sigma
  int* rotated = nullptr;     // Jacobi sweep flags
  // deterministic QRCP (level-3 reflection blocking)
  double* vn1 = nullptr;      // n
  double* vn2 = nullptr;      // n
  int* redo = nullptr;        // n
  double* ys = nullptr;       // m
  double* dots = nullptr;     // kQrcp3Chunks x n
  long long* qcand = nullptr; // 2 per SM
  double* npart = nullptr;    // 1 per SM
  int* ctl = nullptr;         // 4
  // mixed precision (FP32 storage)
  float* omega32 = nullptr;   // l x m
  float* B32 = nullptr;       // l x n
  float* permbuf32 = nullptr; // m x 2b
  double* P64 = nullptr;      // m x b FP64 panel
  float* Y32 = nullptr;       // m x b explicit reflectors
  float* T32 = nullptr;       // b x b
  float* Z32 = nullptr;       // b x n
  float* W32 = nullptr;       // b x n
  double* R12 = nullptr;      // b x n FP64 copy of the new rows of R
  float* tcpart = nullptr;    // split-K partial sums (hi and lo per split)
  size_t tccap = 0;
  __nv_bfloat16* tslA = nullptr;  // bfloat16 slices of op(A) rows
  size_t tslcapA = 0;
  __nv_bfloat16* tslB = nullptr;  // bfloat16 slices of op(B) columns
  size_t tslcapB = 0;
  // FP64 emulation on the tensor cores: operand slices and exponents
  __nv_bfloat16* slA = nullptr;
  size_t slcapA = 0;
  __nv_bfloat16* slB = nullptr;
  size_t slcapB = 0;
  int* exA = nullptr;  // exponents of slA's rows (also of the mixed modes' R12 slices)
  int* exB = nullptr;  // exponents of slB's rows (also of the mixed modes' W11 slices)
  size_t bytes = 0;
};

struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = align_up(off);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

Work carve(char op, int64_t m, int64_t n, int64_t k, int b, int p, int sms, char* base,
           bool emul = false) {
  Work w;
  Carver c{base};
  const int64_t ell = b + p;
  const int64_t bb = b;
  if (op != 'Q' && op != 'X' && op != 'P') {
    w.omega = c.take<double>((size_t)ell * m);
    w.B = c.take<double>((size_t)ell * n);
    w.swaps = c.take<int64_t>(bb);
    w.map = c.take<int64_t>(1 + 10 * bb);
    const int64_t prow = (op == 'R') ? m : k;
    w.permbuf = c.take<double>((size_t)std::max<int64_t>(prow, 1) * 2 * bb);
    w.cand = c.take<double>((size_t)2 * sms * 4);
    w.candcol = c.take<double>((size_t)2 * sms * ell);
    w.W11 = c.take<double>((size_t)bb * bb);
  }
  w.ppart = c.take<double>(rq::panel_partial_doubles(sms, b));
  w.rowj = c.take<double>(2 * bb);
  w.T = c.take<double>((size_t)bb * bb);
  const int64_t zc = std::max(n, k);
  w.Z = c.take<double>((size_t)bb * zc);
  w.W = c.take<double>((size_t)bb * zc);
  // split-K partial sums: up to ~20 splits of a b x max(n, k) product
  w.skcap = std::max((size_t)4 * sms * 4096, (size_t)20 * bb * (size_t)zc) + 4096;
  w.skpart = c.take<double>(w.skcap);
  if (op == 'P') {
    w.vn1 = c.take<double>(n);
    w.vn2 = c.take<double>(n);
    w.redo = c.take<int>(n);
    w.ys = c.take<double>(m);
    w.dots = c.take<double>((size_t)rq::kQrcp3Chunks * n);
    w.qcand = c.take<long long>((size_t)2 * sms);
    w.npart = c.take<double>(sms);
    w.ctl = c.take<int>(4);
  }
  if (op == 'T' || op == 'U') {
    w.Wt = c.take<double>((size_t)k * n);
    w.Ahat = c.take<double>((size_t)m * bb);
    w.YY = c.take<double>((size_t)bb * k);
    w.OY = c.take<double>((size_t)ell * k);
  }
  if (op == 'U') {
    w.Yk = c.take<double>((size_t)m * k);
    w.Rk = c.take<double>((size_t)k * n);
    w.jpvt = c.take<int64_t>(n);
    w.tau = c.take<double>(k);
    w.tau2 = c.take<double>(k);
    w.Tall = c.take<double>((size_t)((k + b - 1) / b) * bb * bb);
    w.F = c.take<double>((size_t)std::max(m, n) * k);
    w.svd = c.take<double>((size_t)5 * k * k + k);
    w.rotated = c.take<int>(rq::kJacobiMaxSweeps);
  } else if (op == 'Q') {
    w.Tall = nullptr;
  } else if (op == 'V') {
    // mixed-precision TRQRCP
    w.omega32 = c.take<float>((size_t)ell * m);
    w.B32 = c.take<float>((size_t)ell * n);
    w.permbuf32 = c.take<float>((size_t)std::max<int64_t>(k, 1) * 2 * bb);
    w.P64 = c.take<double>((size_t)m * bb);
    w.Y32 = c.take<float>((size_t)m * bb);  // A_hat
    w.T32 = c.take<float>((size_t)bb * bb);
    w.Z32 = c.take<float>((size_t)bb * n);
    w.W32 = c.take<float>((size_t)k * n);   // W^T
    w.Wt = c.take<double>((size_t)bb * k);  // Y2^T Y1 as floats (reinterpreted)
    w.R12 = c.take<double>((size_t)bb * n);
    w.tccap = (size_t)16 * bb * n;
    w.tcpart = c.take<float>(w.tccap);
    // the largest split-BF16 products: (b x m)(m x n) and (m x k)(k x b)
    w.tslcapA = std::max(rq::tc_slice_elems(bb, m, 3),
                         std::max(rq::tc_slice_elems(m, k, 3), rq::tc_slice_elems(ell, m, 1)));
    w.tslcapB = std::max(rq::tc_slice_elems(n, m, 3), rq::tc_slice_elems(k, m, 3));
    w.tslA = c.take<__nv_bfloat16>(w.tslcapA);
    w.tslB = c.take<__nv_bfloat16>(w.tslcapB);
    w.exA = c.take<int>(n);
    w.exB = c.take<int>(bb);
  } else if (op == 'G') {
    // split-BF16 GEMM of op(A) (m x k) and op(B) (k x n)
    w.tccap = (size_t)32 * (size_t)std::min<int64_t>(m * n, (int64_t)sms * 128 * 128);
    w.tcpart = c.take<float>(w.tccap);
    w.tslcapA = rq::tc_slice_elems(m, k, 3);
    w.tslcapB = rq::tc_slice_elems(n, k, 3);
    w.tslA = c.take<__nv_bfloat16>(w.tslcapA);
    w.tslB = c.take<__nv_bfloat16>(w.tslcapB);
  } else if (op == 'X') {
    // slices of op(A) (m rows) and op(B)^T (n rows), K = k
    w.slA = c.take<__nv_bfloat16>(rq::oz_slice_elems(m, k));
    w.slB = c.take<__nv_bfloat16>(rq::oz_slice_elems(n, k));
    w.exA = c.take<int>(m);
    w.exB = c.take<int>(n);
  } else if (op == 'M') {
    w.omega32 = c.take<float>((size_t)ell * m);
    w.B32 = c.take<float>((size_t)ell * n);
    w.permbuf32 = c.take<float>((size_t)m * 2 * bb);
    w.P64 = c.take<double>((size_t)m * bb);
    w.Y32 = c.take<float>((size_t)m * bb);
    w.T32 = c.take<float>((size_t)bb * bb);
    w.Z32 = c.take<float>((size_t)bb * n);
    w.W32 = c.take<float>((size_t)bb * n);
    w.R12 = c.take<double>((size_t)bb * n);
    w.tccap = (size_t)16 * bb * n;
    w.tcpart = c.take<float>(w.tccap);
    // the largest split-BF16 products: (b x m)(m x n) and (m x b)(b x n)
    w.tslcapA = std::max(rq::tc_slice_elems(bb, m, 3),
                         std::max(rq::tc_slice_elems(m, bb, 3), rq::tc_slice_elems(ell, m, 1)));
    w.tslcapB = rq::tc_slice_elems(n, m, 3);
    w.tslA = c.take<__nv_bfloat16>(w.tslcapA);
    w.tslB = c.take<__nv_bfloat16>(w.tslcapB);
    w.exA = c.take<int>(n);
    w.exB = c.take<int>(bb);
  }
  if (emul && (op == 'R' || op == 'Q')) {
    // slices of the trailing matrix A2^T (n rows of m) and of Y, W^T, and W^T itself
    w.slcapA = rq::oz_slice_elems(n, m);
    w.slA = c.take<__nv_bfloat16>(w.slcapA);
    // Y sliced twice: b rows of m (as op(B) of Z^T), m rows of b (as op(A) of the update)
    // (and the l x m Omega of the sketch)
    w.slcapB = std::max(rq::oz_slice_elems(std::max<int64_t>(bb, ell), m),
                        rq::oz_slice_elems(m, bb));
    w.slB = c.take<__nv_bfloat16>(w.slcapB);
    w.exA = c.take<int>(std::max(n, m));
    w.exB = c.take<int>(std::max(n, m));
  }
  w.bytes = align_up(c.off) + 256;
  return w;
}

struct Call {
  rqrcp_handle_t h;
  Work w;
  cudaStream_t st;
  int* status;
  int* flag;
  rq::GridBarrier* bar;
};

enum Phase { PH_SKETCH = 0, PH_SAMPLE, PH_PERM, PH_PANEL, PH_TRAIL, PH_SUPD, PH_TRQ, PH_OTHER };

// Brackets a phase region with CUDA events when profiling is on and makes it
// the phase that launch counts are charged to.
struct PhaseScope {
  rqrcp_handle_t h;
  int prev;
  size_t pair = (size_t)-1;
  PhaseScope(rqrcp_handle_t hh, int ph, double flops) : h(hh), prev(hh->cur_phase) {
    h->cur_phase = ph;
    if (!h->prof) return;
    h->flops[ph] += flops;
    if (h->events.size() < 2 * (h->ev_used + 1)) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return;
      }
      h->events.push_back(a);
      h->events.push_back(b);
      h->ev_phase.push_back(ph);
    }
    pair = h->ev_used++;
    h->ev_phase[pair] = ph;
    cudaEventRecord(h->events[2 * pair], h->stream);
  }
  ~PhaseScope() {
    if (pair != (size_t)-1) cudaEventRecord(h->events[2 * pair + 1], h->stream);
    h->cur_phase = prev;
  }
};

void count_launch(rqrcp_handle_t h, int n) {
  h->launch_total += n;
  if (h->prof) h->launches[h->cur_phase] += n;
}

#define CK(expr)                                              \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) {                                  \
      cl.h->err = std::string(#expr) + ": " + cudaGetErrorString(e_); \
      return RQRCP_ERR_CUDA;                                  \
    }                                                         \
  } while (0)

// CK for a launcher that enqueues n kernels
#define CKL(n, expr)                 \
  do {                               \
    CK(expr);                        \
    count_launch(cl.h, (n));         \
  } while (0)

cudaError_t gemm(Call& cl, char ta, char tb, int amode, int64_t M, int64_t N, int64_t K,
                 double alpha, const double* A, int64_t lda, const double* B, int64_t ldb,
                 double beta, double* C, int64_t ldc, const int* gate = nullptr, int gate_run = 0,
                 const int64_t* bcols = nullptr) {
  GemmArgs g{ta, tb, amode, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, gate, gate_run, bcols};
  int s = rq::gemm_pick_splits(M, N, K, cl.h->num_sms);
  while (s > 1 && (size_t)s * M * N > cl.w.skcap) --s;
  if (M > 0 && N > 0) count_launch(cl.h, s > 1 && K > 0 ? 2 : 1);
  return rq::launch_gemm(g, s, cl.w.skpart, cl.st);
}

cudaError_t tcgemm(Call& cl, char ta, char tb, int64_t M, int64_t N, int64_t K, float alpha,
                   const float* A, int64_t lda, const float* B, int64_t ldb, float beta, float* C,
                   int64_t ldc, int slices, const int64_t* bcols = nullptr) {
  rq::TcGemmArgs g{ta,     tb,        M,         N,         K,          alpha,
                   A,      lda,       B,         ldb,       beta,       C,
                   ldc,    cl.status, bcols,     cl.w.tslA, cl.w.tslcapA, cl.w.tslB,
                   cl.w.tslcapB, cl.w.tcpart, cl.w.tccap, cl.h->num_sms};
  count_launch(cl.h, rq::tc_launches(M, N, K, cl.h->num_sms, cl.w.tcpart ? cl.w.tccap : 0));
  return rq::launch_tc_gemm(g, slices, cl.st);
}

int ensure(rqrcp_handle_t h, size_t bytes) {
  if (h->ws_bytes >= bytes) return RQRCP_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && h->ws) e = cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_bytes = 0;
  if (e == cudaSuccess) e = cudaMalloc(&h->ws, bytes);
  if (e != cudaSuccess) {
    h->ws = nullptr;
    h->err = std::string("workspace: ") + cudaGetErrorString(e);
    return RQRCP_ERR_ALLOC;
  }
  h->ws_bytes = bytes;
  return RQRCP_OK;
}

int begin(rqrcp_handle_t h, char op, int64_t m, int64_t n, int64_t k, int b, int p, Call* cl) {
  const bool emul = h->fp64_emulation != 0;
  Work sz = carve(op, m, n, k, b, p, h->num_sms, nullptr, emul);
  int r = ensure(h, sz.bytes);
  if (r != RQRCP_OK) return r;
  cl->h = h;
  cl->w = carve(op, m, n, k, b, p, h->num_sms, h->ws, emul);
  cl->st = h->stream;
  cl->status = h->state;
  cl->flag = h->state + 1;
  cl->bar = reinterpret_cast<rq::GridBarrier*>(reinterpret_cast<char*>(h->state) + 64);
  return RQRCP_OK;
}

// ---------------------------------------------------------------- blocks
int sample_step(Call& cl, double* Bblk, int ell, int64_t nc, int bJ, int f32 = 0) {
  double fl = 0.0;
  for (int i = 0; i < bJ && i < ell; ++i) fl += 4.0 * (ell - i) * (double)(nc - i - 1);
  PhaseScope ps(cl.h, PH_SAMPLE, fl);
  rq::SampleQrcpArgs a{Bblk, ell, ell, nc, bJ, cl.w.swaps, cl.w.cand, cl.w.candcol, cl.bar,
                       cl.status};
  a.f32 = f32;
  CKL(1, rq::launch_sample_qrcp(a, cl.h->num_sms, cl.st));
  return RQRCP_OK;
}

int panel_step(Call& cl, double* P, int64_t ld, int64_t mJ, int bJ, double* tau, double* T,
               int round_f32 = 0) {
  const double b = bJ, m = (double)mJ;
  PhaseScope ps(cl.h, PH_PANEL, 2.0 * m * b * b - 2.0 * b * b * b / 3.0 + m * b * b + b * b * b / 3.0);
  rq::PanelArgs a{P, ld, mJ, bJ, tau, T, cl.w.ppart, cl.w.rowj, cl.bar, cl.status, round_f32};
  CKL(1, rq::launch_panel(a, cl.h->num_sms, cl.st));
  return RQRCP_OK;
}

int swaps_step(Call& cl, double* A, int64_t lda, int64_t rows, int64_t col0, int bJ, int64_t* jpvt) {
  PhaseScope ps(cl.h, PH_PERM, 0.0);
  CKL(3, rq::launch_apply_swaps(A, lda, rows, col0, cl.w.swaps, bJ, jpvt, cl.w.map, cl.w.permbuf,
                                cl.st));
  return RQRCP_OK;
}

// The trailing update with its two large products on the BF16 tensor cores
// (FP64-accurate slicing, oz_gemm.cu): Z^T = A2^T Y (K = mJ), W^T = Z^T T in
// native FP64 (small), A2 -= Y (W^T)^T (K = bJ).
int trailing_update_emulated(Call& cl, const double* P, int64_t ld, int64_t mJ, int bJ,
                             const double* T, double* A2, int64_t n2) {
  Work& w = cl.w;
  double* Zt = w.Z;  // n2 x bJ, ld n2
  double* Wt = w.W;  // n2 x bJ, ld n2
  CKL(rq::oz_slice_launches(true, mJ),
      rq::launch_oz_slice(A2, ld, true, 0, n2, mJ, w.slA, w.exA, cl.st));
  CKL(rq::oz_slice_launches(true, mJ),
      rq::launch_oz_slice(P, ld, true, 1, bJ, mJ, w.slB, w.exB, cl.st));
  float* part = reinterpret_cast<float*>(w.skpart);
  const size_t pcap = 2 * w.skcap;
  rq::OzGemmArgs z{n2,   bJ,      rq::oz_kpad(mJ), w.slA,     w.exA, w.slB, w.exB, 1.0, 0.0,
                   Zt,   n2,      cl.status,       part,      pcap,  cl.h->num_sms};
  CKL(rq::oz_launches(n2, bJ, z.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(z, cl.st));
  CK(gemm(cl, 'N', 'N', 0, n2, bJ, bJ, 1.0, Zt, n2, T, bJ, 0.0, Wt, n2));
  CKL(rq::oz_slice_launches(false, bJ),
      rq::launch_oz_slice(P, ld, false, 1, mJ, bJ, w.slB, w.exB, cl.st));
  CKL(rq::oz_slice_launches(false, bJ),
      rq::launch_oz_slice(Wt, n2, false, 0, n2, bJ, w.slA, w.exA, cl.st));
  rq::OzGemmArgs u{mJ, n2, rq::oz_kpad(bJ), w.slB,  w.exB, w.slA,        w.exA, -1.0, 1.0,
                   A2, ld, cl.status,       part,   pcap,  cl.h->num_sms};
  CKL(rq::oz_launches(mJ, n2, u.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(u, cl.st));
  return RQRCP_OK;
}

// Eq. (3)'s product S12 -= W11 R12 (W11 bJ x bJ, R12 bJ x n2 with leading
// dimension ldr, S12 bJ x n2 with leading dimension lds): FP64-accurate slice
// products on the tensor cores (oz_gemm.cu) when the slice buffers given hold
// both operands, else the FP64 GEMM gated off by the re-sample flag.  The
// tensor-core product is not gated: W11 = 0 when the flag is raised, so it
// leaves S12 unchanged.
int sample_update_product(Call& cl, const double* W11, int bJ, const double* R12, int64_t ldr,
                          int64_t n2, double* S12, int64_t lds, __nv_bfloat16* slW, size_t capW,
                          int* exW, __nv_bfloat16* slR, size_t capR, int* exR) {
  if (n2 <= 0) return RQRCP_OK;
  if (slW != nullptr && slR != nullptr && exW != nullptr && exR != nullptr &&
      rq::oz_slice_elems(bJ, bJ) <= capW && rq::oz_slice_elems(n2, bJ) <= capR) {
    CKL(rq::oz_slice_launches(false, bJ),
        rq::launch_oz_slice(W11, bJ, false, 0, bJ, bJ, slW, exW, cl.st));
    CKL(rq::oz_slice_launches(true, bJ),
        rq::launch_oz_slice(R12, ldr, true, 0, n2, bJ, slR, exR, cl.st));
    float* part = reinterpret_cast<float*>(cl.w.skpart);
    const size_t pcap = 2 * cl.w.skcap;
    rq::OzGemmArgs su{bJ,  n2,  rq::oz_kpad(bJ), slW,       exW,  slR,  exR,  -1.0,
                      1.0, S12, lds,             cl.status, part, pcap, cl.h->num_sms};
    CKL(rq::oz_launches(bJ, n2, su.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(su, cl.st));
    return RQRCP_OK;
  }
  CK(gemm(cl, 'N', 'N', 2, bJ, n2, bJ, -1.0, W11, bJ, R12, ldr, 1.0, S12, lds, cl.flag, 0));
  return RQRCP_OK;
}

// A2 <- Q^T A2 with Q = I - Y T Y^T; Y = unit-lower part of P (mJ x bJ, ld),
// A2 mJ x n2 (ld).  Rows 0..bJ-1 of the result are R12.
int trailing_update(Call& cl, const double* P, int64_t ld, int64_t mJ, int bJ, const double* T,
                    double* A2, int64_t n2) {
  if (n2 <= 0) return RQRCP_OK;
  PhaseScope ps(cl.h, PH_TRAIL, 4.0 * (double)mJ * (double)n2 * bJ + 2.0 * bJ * bJ * (double)n2);
  if (cl.w.slA != nullptr && bJ <= 64) return trailing_update_emulated(cl, P, ld, mJ, bJ, T, A2, n2);
  CK(gemm(cl, 'T', 'N', 1, bJ, n2, mJ, 1.0, P, ld, A2, ld, 0.0, cl.w.Z, bJ));
  CK(gemm(cl, 'T', 'N', 0, bJ, n2, bJ, 1.0, T, bJ, cl.w.Z, bJ, 0.0, cl.w.W, bJ));
  CK(gemm(cl, 'N', 'N', 1, mJ, n2, bJ, -1.0, P, ld, cl.w.W, bJ, 1.0, A2, ld));
  return RQRCP_OK;
}

// Unpivoted blocked QR of F (M x N, ldf) in place; T of block J stored at
// Tall + J*b*b when Tall != nullptr.
int qr_core(Call& cl, int64_t M, int64_t N, double* F, int64_t ldf, int b, double* tau,
            double* Tall) {
  const int64_t k = std::min(M, N);
  int J = 0;
  for (int64_t j0 = 0; j0 < k; j0 += b, ++J) {
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    double* P = F + j0 + j0 * ldf;
    double* T = Tall ? Tall + (size_t)J * b * b : cl.w.T;
    int r = panel_step(cl, P, ldf, M - j0, bJ, tau + j0, T);
    if (r) return r;
    r = trailing_update(cl, P, ldf, M - j0, bJ, T, F + j0 + (j0 + bJ) * ldf, N - j0 - bJ);
    if (r) return r;
  }
  return RQRCP_OK;
}

// Q (M x K, ldq) = first K columns of H_0 ... H_{K-1} from reflectors in F
// (M x K, ldf) and the block factors Tall.
int orgqr_core(Call& cl, int64_t M, int64_t K, const double* F, int64_t ldf, int b,
               const double* Tall, double* Q, int64_t ldq) {
  // Q starts as the first K columns of the identity
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_eye(Q, M, K, ldq, cl.st));
  }
  PhaseScope ps(cl.h, PH_TRQ, 4.0 * (double)M * (double)K * (double)K);
  const int nblk = (int)((K + b - 1) / b);
  for (int J = nblk - 1; J >= 0; --J) {
    const int64_t j0 = (int64_t)J * b;
    const int bJ = (int)std::min<int64_t>(b, K - j0);
    const double* P = F + j0 + j0 * ldf;
    const double* T = Tall + (size_t)J * b * b;  // ld bJ
    const int64_t nc = K - j0;                   // columns < j0 of Q are still e_i
    double* Qb = Q + j0 + j0 * ldq;
    CK(gemm(cl, 'T', 'N', 1, bJ, nc, M - j0, 1.0, P, ldf, Qb, ldq, 0.0, cl.w.Z, bJ));
    CK(gemm(cl, 'N', 'N', 0, bJ, nc, bJ, 1.0, T, bJ, cl.w.Z, bJ, 0.0, cl.w.W, bJ));
    CK(gemm(cl, 'N', 'N', 1, M - j0, nc, bJ, -1.0, P, ldf, cl.w.W, bJ, 1.0, Qb, ldq));
  }
  return RQRCP_OK;
}

bool sizes_fit(int num_sms, int64_t m, int64_t n, int b, int ell) {
  if (b > kMaxB || ell > kMaxEll) return false;
  if (ell > 0 && !rq::sample_qrcp_fits(ell, n, num_sms)) return false;
  if (!rq::panel_fits(m, b, num_sms)) return false;
  return true;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

int rqrcp_create(rqrcp_handle_t* handle, void* cuda_stream) {
  if (!handle) return -1;
  *handle = nullptr;
  rqrcp_handle_s* h = new rqrcp_handle_s();
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
  h->dev_sms = h->num_sms;
  if (e == cudaSuccess) e = cudaMalloc(&h->state, 256);
  if (e == cudaSuccess) e = cudaMemset(h->state, 0, 256);
  if (e != cudaSuccess) {
    if (h->state) cudaFree(h->state);
    delete h;
    return RQRCP_ERR_CUDA;
  }
  *handle = h;
  return RQRCP_OK;
}

int rqrcp_destroy(rqrcp_handle_t h) {
  if (!h) return -1;
  cudaStreamSynchronize(h->stream);
  if (h->ring_host) {
    // a server launch still running exits once it sees the stop word
    reinterpret_cast<rq::RequestRing*>(h->ring_host)->stop = 1;
    cudaStreamSynchronize(h->stream);
    cudaFreeHost(h->ring_host);
  }
  if (h->bt_scratch) cudaFree(h->bt_scratch);
  if (h->bt_ctl) cudaFree(h->bt_ctl);
  if (h->bt_table) cudaFree(h->bt_table);
  if (h->bt_stage) cudaFreeHost(h->bt_stage);
  if (h->bt_copy_ev) cudaEventDestroy(h->bt_copy_ev);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  if (h->io_st) cudaStreamSynchronize(h->io_st);
  for (cudaEvent_t e : h->io_ev) cudaEventDestroy(e);
  if (h->io_st) cudaStreamDestroy(h->io_st);
  if (h->io_jpvt) cudaFree(h->io_jpvt);
  if (h->io_tau) cudaFree(h->io_tau);
  if (h->ws) cudaFree(h->ws);
  if (h->state) cudaFree(h->state);
  delete h;
  return RQRCP_OK;
}

int rqrcp_set_stream(rqrcp_handle_t h, void* cuda_stream) {
  if (!h) return -1;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return RQRCP_OK;
}

size_t rqrcp_workspace_bytes(char op, int64_t m, int64_t n, int64_t k, int b, int p) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (op == 'R' || op == 'Q' || op == 'P' || op == 'M') k = std::min(m, n);
  if (b > k) b = (int)std::max<int64_t>(k, 1);
  return carve(op, m, n, k, b, p, sms, nullptr).bytes;
}

int rqrcp_reserve(rqrcp_handle_t h, char op, int64_t m, int64_t n, int64_t k, int b, int p) {
  if (!h) return -1;
  if (op == 'R' || op == 'Q' || op == 'P' || op == 'M') k = std::min(m, n);
  if (b > k) b = (int)std::max<int64_t>(k, 1);
  return ensure(h, carve(op, m, n, k, b, p, h->num_sms, nullptr, h->fp64_emulation != 0).bytes);
}

int rqrcp_set_option(rqrcp_handle_t h, int option, int value) {
  if (!h) return -1;
  if (option == RQRCP_OPT_FP64_EMULATION) {
    h->fp64_emulation = value != 0;
    return RQRCP_OK;
  }
  if (option == RQRCP_OPT_RESAMPLE) {
    h->resample = value != 0;
    return RQRCP_OK;
  }
  if (option == RQRCP_OPT_BATCH_TEAM) {
    if (value != 8 && value != 16 && value != 32) return -3;
    if (value != h->bt_G) {
      // the team scratch layout depends on the team size: rebuilt on next use
      cudaStreamSynchronize(h->stream);
      if (h->bt_scratch) cudaFree(h->bt_scratch);
      h->bt_scratch = nullptr;
      h->bt_teams = 0;
      h->bt_lim = rq::BatchLimits{};
      h->bt_G = value;
    }
    return RQRCP_OK;
  }
  if (option == RQRCP_OPT_TEST_BARRIER_TIMEOUT) {
    h->test_timeout = value != 0;
    return RQRCP_OK;
  }
  if (option == RQRCP_OPT_MAX_SMS) {
    if (value < 0) return -3;
    h->num_sms = (value == 0 || value > h->dev_sms) ? h->dev_sms : value;
    return RQRCP_OK;
  }
  return -2;
}

int rqrcp_sync_info(rqrcp_handle_t h, int* info) {
  if (!h) return -1;
  if (!info) return -2;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) e = cudaMemcpy(info, h->state, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(h->state, 0, sizeof(int));
  if (e != cudaSuccess) {
    h->err = std::string("sync_info: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  return RQRCP_OK;
}

const char* rqrcp_last_error(rqrcp_handle_t h) { return h ? h->err.c_str() : ""; }

const char* rqrcp_status_string(int code) {
  switch (code) {
    case RQRCP_OK: return "ok";
    case RQRCP_ERR_CUDA: return "CUDA runtime error";
    case RQRCP_ERR_ALLOC: return "workspace allocation failed";
    case RQRCP_ERR_UNSUPPORTED: return "size outside the supported limits";
    case RQRCP_ERR_BATCH: return "a problem of the batch failed its checks";
    case RQRCP_ERR_BUSY: return "the request ring is full: poll and retry";
    case RQRCP_INFO_NONFINITE: return "non-finite input";
    case RQRCP_INFO_RESAMPLED: return "singular R11: sample re-drawn";
    case RQRCP_INFO_TIMEOUT: return "device wait timed out";
    default: return code < 0 ? "invalid argument" : "unknown";
  }
}

int rqrcp_gaussian(rqrcp_handle_t h, uint64_t seed, uint32_t stream_id, int64_t rows, int64_t cols,
                   double* dOut, int64_t ldo) {
  if (!h) return -1;
  if (rows < 0) return -4;
  if (cols < 0) return -5;
  if (!dOut && rows * cols > 0) return -6;
  if (ldo < std::max<int64_t>(1, rows)) return -7;
  Call cl{};
  cl.h = h;
  cl.st = h->stream;
  PhaseScope ps(h, PH_SKETCH, 0.0);
  CKL(1, rq::launch_gaussian(seed, stream_id, rows, cols, dOut, ldo, nullptr, cl.st));
  return RQRCP_OK;
}

int rqrcp_sketch(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda, int ell,
                 uint64_t seed, double* dB, int64_t ldb) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (ell < 1) return -6;
  if (!dB) return -8;
  if (ldb < ell) return -9;
  Call cl;
  int r = begin(h, 'S', m, n, 1, 1, ell - 1, &cl);
  if (r) return r;
  PhaseScope ps(h, PH_SKETCH, 2.0 * ell * (double)m * (double)n);
  CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, cl.w.omega, ell, nullptr, cl.st));
  CK(gemm(cl, 'N', 'N', 0, ell, n, m, 1.0, cl.w.omega, ell, dA, lda, 0.0, dB, ldb));
  return RQRCP_OK;
}

int rqrcp_sample_qrcp(rqrcp_handle_t h, int ell, int64_t nc, int steps, double* dB, int64_t ldb,
                      int64_t* d_swaps) {
  if (!h) return -1;
  if (ell < 1 || ell > kMaxEll) return -2;
  if (nc < 1) return -3;
  if (steps < 1 || steps > ell || steps > nc) return -4;
  if (!dB) return -5;
  if (ldb < ell) return -6;
  if (!d_swaps) return -7;
  if (!rq::sample_qrcp_fits(ell, nc, h->num_sms)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'S', ell, nc, 1, 1, ell - 1, &cl);
  if (r) return r;
  double fl = 0.0;
  for (int i = 0; i < steps; ++i) fl += 4.0 * (ell - i) * (double)(nc - i - 1);
  PhaseScope ps(cl.h, PH_SAMPLE, fl);
  rq::SampleQrcpArgs a{dB, ldb, ell, nc, steps, d_swaps, cl.w.cand, cl.w.candcol, cl.bar,
                       cl.status};
  a.phantom = h->test_timeout ? 1 : 0;
  CKL(1, rq::launch_sample_qrcp(a, cl.h->num_sms, cl.st));
  return RQRCP_OK;
}

// Host buffers of rqrcp_factor_host and the copy stream that moves them while
// the factorization runs on the handle's stream.
struct HostIO {
  const double* hA;
  int64_t ldha;
  double* hF;
  int64_t ldhf;
  // device-side addresses of hA / hF when they are page-locked and mapped
  // (the copies are then made by a kernel), else nullptr (copy engine)
  const double* mA;
  double* mF;
  int64_t* h_jpvt;
  double* h_tau;
  cudaStream_t cs;
  cudaEvent_t* ev;
  int nev;
  int used;
  int64_t chunk;    // columns per upload
  int64_t group;    // columns per download
  int64_t copied;   // columns [0, copied) downloaded (enqueued)
  cudaEvent_t next() { return ev[used++ % nev]; }
};

// Enqueue on the copy stream, after everything enqueued so far on the compute
// stream, the download of the final columns [io.copied, upto).
cudaError_t io_download(Call& cl, HostIO& io, const double* dA, int64_t lda, int64_t m,
                        int64_t upto) {
  if (upto <= io.copied) return cudaSuccess;
  cudaEvent_t e = io.next();
  cudaError_t r = cudaEventRecord(e, cl.st);
  if (r == cudaSuccess) r = cudaStreamWaitEvent(io.cs, e, 0);
  if (r == cudaSuccess && io.mF != nullptr) {
    r = rq::launch_copy_mapped(dA + io.copied * lda, lda, io.mF + io.copied * io.ldhf, io.ldhf,
                               m, upto - io.copied, io.cs);
    if (r == cudaSuccess) count_launch(cl.h, 1);
  } else if (r == cudaSuccess) {
    r = cudaMemcpy2DAsync(io.hF + io.copied * io.ldhf, io.ldhf * sizeof(double),
                          dA + io.copied * lda, lda * sizeof(double), m * sizeof(double),
                          upto - io.copied, cudaMemcpyDeviceToHost, io.cs);
  }
  io.copied = upto;
  return r;
}

// Device-side address of page-locked, mapped host memory; nullptr for
// pageable memory (or anything else).
const void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

int rqrcp_factor_core(Call& cl, int64_t m, int64_t n, double* dA, int64_t lda, int b, int p,
                      uint64_t seed, int64_t* d_jpvt, double* d_tau, HostIO* io) {
  rqrcp_handle_t h = cl.h;
  const int64_t k = std::min(m, n);
  const int ell = b + p;
  int r;
  Work& w = cl.w;
  if (io != nullptr) {
    // the copy stream starts after the work already on the compute stream
    cudaEvent_t e = io->next();
    CK(cudaEventRecord(e, cl.st));
    CK(cudaStreamWaitEvent(io->cs, e, 0));
  }
  // Alg. 4: Omega^[0] and the initial sample B^[0] = Omega^[0] A^[0]
  {
    PhaseScope ps(cl.h, PH_SKETCH, 2.0 * ell * (double)m * (double)n);
    if (io != nullptr && w.slA != nullptr) {
      // the sliced sketch needs all of A: upload first
      if (io->mA != nullptr)
        CKL(1, rq::launch_copy_mapped(io->mA, io->ldha, dA, lda, m, n, io->cs));
      else
        CK(cudaMemcpy2DAsync(dA, lda * sizeof(double), io->hA, io->ldha * sizeof(double),
                             m * sizeof(double), n, cudaMemcpyHostToDevice, io->cs));
      cudaEvent_t e = io->next();
      CK(cudaEventRecord(e, io->cs));
      CK(cudaStreamWaitEvent(cl.st, e, 0));
    }
    if (w.slA != nullptr) {
      // FP64-accurate product on the tensor cores: Omega stored transposed so
      // that its rows are contiguous for the slicing pass
      CKL(1, rq::launch_gaussian_t(seed, kOmegaStream, ell, m, w.omega, m, cl.st));
      CKL(rq::oz_slice_launches(true, m),
          rq::launch_oz_slice(w.omega, m, true, 0, ell, m, w.slB, w.exB, cl.st));
      CKL(rq::oz_slice_launches(true, m),
          rq::launch_oz_slice(dA, lda, true, 0, n, m, w.slA, w.exA, cl.st));
      float* part = reinterpret_cast<float*>(w.skpart);
      const size_t pcap = 2 * w.skcap;
      rq::OzGemmArgs sk{ell, n,  rq::oz_kpad(m), w.slB, w.exB, w.slA,         w.exA, 1.0, 0.0,
                        w.B, ell, cl.status,     part,  pcap,  cl.h->num_sms};
      CKL(rq::oz_launches(ell, n, sk.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(sk, cl.st));
    } else if (io != nullptr) {
      // upload in column chunks; each chunk's share of the sketch starts as
      // soon as it has landed
      CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, w.omega, ell, nullptr, cl.st));
      for (int64_t c0 = 0; c0 < n; c0 += io->chunk) {
        const int64_t nc = std::min(io->chunk, n - c0);
        if (io->mA != nullptr)
          CKL(1, rq::launch_copy_mapped(io->mA + c0 * io->ldha, io->ldha, dA + c0 * lda, lda, m,
                                        nc, io->cs));
        else
          CK(cudaMemcpy2DAsync(dA + c0 * lda, lda * sizeof(double), io->hA + c0 * io->ldha,
                               io->ldha * sizeof(double), m * sizeof(double), nc,
                               cudaMemcpyHostToDevice, io->cs));
        cudaEvent_t e = io->next();
        CK(cudaEventRecord(e, io->cs));
        CK(cudaStreamWaitEvent(cl.st, e, 0));
        CK(gemm(cl, 'N', 'N', 0, ell, nc, m, 1.0, w.omega, ell, dA + c0 * lda, lda, 0.0,
                w.B + c0 * ell, ell));
      }
    } else {
      CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, w.omega, ell, nullptr, cl.st));
      CK(gemm(cl, 'N', 'N', 0, ell, n, m, 1.0, w.omega, ell, dA, lda, 0.0, w.B, ell));
    }
    CKL(1, rq::launch_iota(d_jpvt, n, cl.st));
  }
  int J = 0;
  for (int64_t j0 = 0; j0 < k; j0 += b) {
    ++J;
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    const int64_t nc = n - j0, n2 = nc - bJ, mJ = m - j0;
    double* Bblk = w.B + j0 * ell;
    // b pivots from the sample; S left in B in the permuted order
    if ((r = sample_step(cl, Bblk, ell, nc, bJ))) return r;
    // permute whole columns of the A/R array and jpvt
    if ((r = swaps_step(cl, dA, lda, m, j0, bJ, d_jpvt))) return r;
    // reflectors and R11 from the new leading columns, then T
    double* P = dA + j0 + j0 * lda;
    if ((r = panel_step(cl, P, lda, mJ, bJ, d_tau + j0, w.T))) return r;
    // R12 and the trailing matrix A^[J]
    if ((r = trailing_update(cl, P, lda, mJ, bJ, w.T, dA + j0 + (j0 + bJ) * lda, n2))) return r;
    if (j0 + bJ < k && h->resample) {
      // Alg. 5 (RSRQRCP): a fresh GIID sample of the updated trailing matrix
      const int64_t mt = m - j0 - bJ;
      double* Bnext = Bblk + (int64_t)bJ * ell;
      const double* At = dA + (j0 + bJ) + (j0 + bJ) * lda;
      PhaseScope ps(cl.h, PH_SUPD, 2.0 * ell * (double)mt * (double)n2);
      if (w.slA != nullptr) {
        CKL(1, rq::launch_gaussian_t(seed, kResampleStreamBase + J, ell, mt, w.omega, mt, cl.st));
        CKL(rq::oz_slice_launches(true, mt),
            rq::launch_oz_slice(w.omega, mt, true, 0, ell, mt, w.slB, w.exB, cl.st));
        CKL(rq::oz_slice_launches(true, mt),
            rq::launch_oz_slice(At, lda, true, 0, n2, mt, w.slA, w.exA, cl.st));
        float* part = reinterpret_cast<float*>(w.skpart);
        const size_t pcap = 2 * w.skcap;
        rq::OzGemmArgs rs{ell,   n2,  rq::oz_kpad(mt), w.slB, w.exB, w.slA,         w.exA, 1.0,
                          0.0,   Bnext, ell,           cl.status, part, pcap,        cl.h->num_sms};
        CKL(rq::oz_launches(ell, n2, rs.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(rs, cl.st));
      } else {
        CKL(1, rq::launch_gaussian(seed, kResampleStreamBase + J, ell, mt, w.omega, ell, nullptr,
                                   cl.st));
        CK(gemm(cl, 'N', 'N', 0, ell, n2, mt, 1.0, w.omega, ell, At, lda, 0.0, Bnext, ell));
      }
    } else if (j0 + bJ < k) {
      PhaseScope ps(cl.h, PH_SUPD, (double)bJ * bJ * bJ / 3.0 + 2.0 * bJ * bJ * (double)n2);
      // Eq. (3): B1 = S12 - S11 R11^{-1} R12, B2 = S22 (in place)
      CKL(1, rq::launch_w11(Bblk, ell, P, lda, bJ, w.W11, cl.flag, cl.status, cl.st));
      double* Bnext = Bblk + (int64_t)bJ * ell;
      // with FP64 emulation on the tensor cores (the re-sample below then
      // overwrites S12 when the flag is raised), else FP64
      if ((r = sample_update_product(cl, w.W11, bJ, dA + j0 + (j0 + bJ) * lda, lda, n2, Bnext, ell,
                                     w.slB, w.slcapB, w.exB, w.slA, w.slcapA, w.exA)))
        return r;
      // exactly singular R11: fresh sample of the trailing matrix (Alg. 5 step)
      const int64_t mt = m - j0 - bJ;
      CKL(1, rq::launch_gaussian(seed, kResampleStreamBase + J, ell, mt, w.omega, ell, cl.flag, cl.st));
      CK(gemm(cl, 'N', 'N', 0, ell, n2, mt, 1.0, w.omega, ell, dA + (j0 + bJ) + (j0 + bJ) * lda,
              lda, 0.0, Bnext, ell, cl.flag, 1));
    }
    // columns [0, j0 + bJ) are final (later blocks only touch and permute
    // trailing columns); after the last block all n are
    if (io != nullptr) {
      const int64_t fin = (j0 + bJ >= k) ? n : j0 + bJ;
      if (fin == n || fin - io->copied >= io->group) CK(io_download(cl, *io, dA, lda, m, fin));
    }
  }
  if (io != nullptr) {
    cudaEvent_t e = io->next();
    CK(cudaEventRecord(e, cl.st));
    CK(cudaStreamWaitEvent(io->cs, e, 0));
    CK(cudaMemcpyAsync(io->h_jpvt, d_jpvt, n * sizeof(int64_t), cudaMemcpyDeviceToHost, io->cs));
    CK(cudaMemcpyAsync(io->h_tau, d_tau, k * sizeof(double), cudaMemcpyDeviceToHost, io->cs));
    // the compute stream completes only after the copies
    e = io->next();
    CK(cudaEventRecord(e, io->cs));
    CK(cudaStreamWaitEvent(cl.st, e, 0));
  }
  return RQRCP_OK;
}

int rqrcp_factor(rqrcp_handle_t h, int64_t m, int64_t n, double* dA, int64_t lda, int b, int p,
                 uint64_t seed, int64_t* d_jpvt, double* d_tau) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (b < 1) return -6;
  if (p < 0) return -7;
  if (!d_jpvt) return -9;
  if (!d_tau) return -10;
  const int64_t k = std::min(m, n);
  if (b > k) b = (int)k;
  if (!sizes_fit(h->num_sms, m, n, b, b + p)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'R', m, n, k, b, p, &cl);
  if (r) return r;
  return rqrcp_factor_core(cl, m, n, dA, lda, b, p, seed, d_jpvt, d_tau, nullptr);
}

int rqrcp_factor_host(rqrcp_handle_t h, int64_t m, int64_t n, const double* hA, int64_t ldha,
                      double* dA, int64_t lda, int b, int p, uint64_t seed, double* hF,
                      int64_t ldhf, int64_t* h_jpvt, double* h_tau) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!hA) return -4;
  if (ldha < m) return -5;
  if (!dA) return -6;
  if (lda < m) return -7;
  if (b < 1) return -8;
  if (p < 0) return -9;
  if (!hF) return -11;
  if (ldhf < m) return -12;
  if (!h_jpvt) return -13;
  if (!h_tau) return -14;
  const int64_t k = std::min(m, n);
  if (b > k) b = (int)k;
  if (!sizes_fit(h->num_sms, m, n, b, b + p)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'R', m, n, k, b, p, &cl);
  if (r) return r;
  cudaError_t e = cudaSuccess;
  if (!h->io_st) e = cudaStreamCreateWithFlags(&h->io_st, cudaStreamNonBlocking);
  while (e == cudaSuccess && h->io_ev.size() < 64) {
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) h->io_ev.push_back(ev);
  }
  if (e == cudaSuccess && h->io_cap < n) {
    // device pivots and tau of the call (grown like the workspace)
    e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->io_st);
    if (h->io_jpvt) cudaFree(h->io_jpvt);
    if (h->io_tau) cudaFree(h->io_tau);
    h->io_jpvt = nullptr;
    h->io_tau = nullptr;
    h->io_cap = 0;
    if (e == cudaSuccess) e = cudaMalloc(&h->io_jpvt, n * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&h->io_tau, n * sizeof(double));
    if (e == cudaSuccess) h->io_cap = n;
  }
  if (e != cudaSuccess) {
    h->err = std::string("rqrcp_factor_host: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  HostIO io{hA,
            ldha,
            hF,
            ldhf,
            static_cast<const double*>(mapped_host(hA)),
            static_cast<double*>(const_cast<void*>(mapped_host(hF))),
            h_jpvt,
            h_tau,
            h->io_st,
            h->io_ev.data(),
            (int)h->io_ev.size(),
            0,
            0,
            0,
            0};
  // 8 upload chunks; downloads every ~n/16 columns, in whole blocks
  io.chunk = std::max<int64_t>(1, (n + 7) / 8);
  io.group = std::max<int64_t>(b, (n + 15) / 16 / b * b);
  return rqrcp_factor_core(cl, m, n, dA, lda, b, p, seed, h->io_jpvt, h->io_tau, &io);
}

int qr_factor(rqrcp_handle_t h, int64_t m, int64_t n, double* dA, int64_t lda, int b,
              double* d_tau) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (b < 1) return -6;
  if (!d_tau) return -7;
  const int64_t k = std::min(m, n);
  if (b > k) b = (int)k;
  if (!sizes_fit(h->num_sms, m, n, b, 0)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'Q', m, n, k, b, 0, &cl);
  if (r) return r;
  return qr_core(cl, m, n, dA, lda, b, d_tau, nullptr);
}

int qrcp_factor(rqrcp_handle_t h, int64_t m, int64_t n, double* dA, int64_t lda, int b,
                int64_t* d_jpvt, double* d_tau) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (b < 1) return -6;
  if (!d_jpvt) return -7;
  if (!d_tau) return -8;
  const int64_t k = std::min(m, n);
  if (b > k) b = (int)k;
  if (b > rq::kQrcp3MaxB) b = rq::kQrcp3MaxB;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    h->err = "qrcp_factor reads each block's length back on the host: not capturable";
    return RQRCP_ERR_UNSUPPORTED;
  }
  Call cl;
  int r = begin(h, 'P', m, n, k, b, 0, &cl);
  if (r) return r;
  Work& w = cl.w;
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_iota(d_jpvt, n, cl.st));
    // every norm starts "to be recomputed": the first block computes them all
    CK(cudaMemsetAsync(w.redo, 1, sizeof(int) * (size_t)n, cl.st));
  }
  int64_t i0 = 0;
  while (i0 < k) {
    const int bJ = (int)std::min<int64_t>(b, k - i0);
    const int64_t mJ = m - i0, nJ = n - i0;
    {
      PhaseScope ps(cl.h, PH_PANEL, 4.0 * (double)mJ * (double)nJ * bJ);
      rq::Qrcp3Args qa{dA,      lda,    m,     n,      i0,     bJ,       w.vn1,   w.vn2,
                       w.redo,  d_jpvt, d_tau, w.W,    w.ys,   w.dots,   w.qcand, w.npart,
                       w.ctl,   cl.bar, cl.status, 0};
      CKL(1, rq::launch_qrcp3_block(qa, cl.h->num_sms, cl.st));
    }
    int ctl[2] = {0, 0};
    CK(cudaMemcpyAsync(ctl, w.ctl, sizeof(ctl), cudaMemcpyDeviceToHost, cl.st));
    CK(cudaStreamSynchronize(cl.st));
    const int nb = ctl[1];
    if (nb < 1 || nb > bJ) break;  // a grid barrier gave up: RQRCP_INFO_TIMEOUT is set
    const int64_t i1 = i0 + nb;
    if (i1 < m && i1 < n) {
      // the delayed block update A22 -= Y W^T
      PhaseScope ps(cl.h, PH_TRAIL, 2.0 * (double)(m - i1) * (double)(n - i1) * nb);
      CK(gemm(cl, 'N', 'T', 0, m - i1, n - i1, nb, -1.0, dA + i1 + i0 * lda, lda, w.W + i1, n,
              1.0, dA + i1 + i1 * lda, lda));
    }
    i0 = i1;
  }
  return RQRCP_OK;
}

namespace {

// Alg. 6 on device buffers; Y (m x k, ldy) and R (k x n, ldr) outputs.
int trqrcp_core(Call& cl, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k, int b,
                int ell, uint64_t seed, int64_t* jpvt, double* tau, double* Y, int64_t ldy,
                double* R, int64_t ldr) {
  Work& w = cl.w;
  int r;
  {
    PhaseScope ps(cl.h, PH_SKETCH, 2.0 * ell * (double)m * (double)n);
    CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, w.omega, ell, nullptr, cl.st));
    CK(gemm(cl, 'N', 'N', 0, ell, n, m, 1.0, w.omega, ell, dA, lda, 0.0, w.B, ell));
  }
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_iota(jpvt, n, cl.st));
    CKL(1, rq::launch_fill(Y, m, k, ldy, 0.0, cl.st));
    CKL(1, rq::launch_fill(R, k, n, ldr, 0.0, cl.st));
    CKL(1, rq::launch_fill(w.Wt, k, n, k, 0.0, cl.st));
  }
  int J = 0;
  for (int64_t j0 = 0; j0 < k; j0 += b) {
    ++J;
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    const int64_t nc = n - j0, n2 = nc - bJ, mJ = m - j0;
    double* Bblk = w.B + j0 * ell;
    if ((r = sample_step(cl, Bblk, ell, nc, bJ))) return r;
    // permute jpvt, prior inner products W^T and completed rows of R
    if ((r = swaps_step(cl, w.Wt, k, j0, j0, bJ, jpvt))) return r;
    if ((r = swaps_step(cl, R, ldr, j0, j0, bJ, nullptr))) return r;
    {
      // selected columns A_hat = A(:, sel) - Y1 W1^T(:, sel), rows j0..m-1
      PhaseScope ps(cl.h, PH_TRQ, 2.0 * (double)mJ * bJ * (double)j0);
      CKL(1, rq::launch_gather_cols(dA, lda, j0, mJ, jpvt + j0, bJ, w.Ahat, m, cl.st));
      if (j0 > 0)
        CK(gemm(cl, 'N', 'N', 0, mJ, bJ, j0, -1.0, Y + j0, ldy, w.Wt + j0 * k, k, 1.0, w.Ahat, m));
    }
    if ((r = panel_step(cl, w.Ahat, m, mJ, bJ, tau + j0, w.T))) return r;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      CKL(1, rq::launch_split_qr(w.Ahat, m, mJ, bJ, j0, Y + j0 * ldy, ldy, R + j0 + j0 * ldr, ldr,
                                 cl.st));
    }
    if (n2 > 0) {
      PhaseScope ps(cl.h, PH_TRQ,
                    2.0 * bJ * (double)mJ * (double)n2 + 2.0 * bJ * (double)mJ * j0 +
                        2.0 * bJ * (double)j0 * (double)n2 + 2.0 * bJ * bJ * (double)n2 +
                        2.0 * bJ * (double)(j0 + bJ) * (double)n2);
      const int64_t* tcols = jpvt + j0 + bJ;
      double* Y2 = Y + j0 + j0 * ldy;  // rows j0.., explicit unit lower
      // W2^T = T2^T (Y2^T A(:, trailing) - (Y2^T Y1) W1^T(:, trailing))
      CK(gemm(cl, 'T', 'N', 0, bJ, n2, mJ, 1.0, Y2, ldy, dA + j0, lda, 0.0, w.Z, bJ, nullptr, 0,
              tcols));
      if (j0 > 0) {
        CK(gemm(cl, 'T', 'N', 0, bJ, j0, mJ, 1.0, Y2, ldy, Y + j0, ldy, 0.0, w.YY, bJ));
        CK(gemm(cl, 'N', 'N', 0, bJ, n2, j0, -1.0, w.YY, bJ, w.Wt + (j0 + bJ) * k, k, 1.0, w.Z, bJ));
      }
      CK(gemm(cl, 'T', 'N', 0, bJ, n2, bJ, 1.0, w.T, bJ, w.Z, bJ, 0.0, w.Wt + j0 + (j0 + bJ) * k, k));
      // new rows of R: A(rows J, trailing) - Y(rows J, :) W^T(:, trailing)
      double* Rrows = R + j0 + (j0 + bJ) * ldr;
      CKL(1, rq::launch_gather_cols(dA, lda, j0, bJ, tcols, n2, Rrows, ldr, cl.st));
      CK(gemm(cl, 'N', 'N', 0, bJ, n2, j0 + bJ, -1.0, Y + j0, ldy, w.Wt + (j0 + bJ) * k, k, 1.0,
              Rrows, ldr));
    }
    if (j0 + bJ < k) {
      PhaseScope ps(cl.h, PH_SUPD, (double)bJ * bJ * bJ / 3.0 + 2.0 * bJ * bJ * (double)n2);
      const double* R11 = R + j0 + j0 * ldr;
      CKL(1, rq::launch_w11(Bblk, ell, R11, ldr, bJ, w.W11, cl.flag, cl.status, cl.st));
      double* Bnext = Bblk + (int64_t)bJ * ell;
      CK(gemm(cl, 'N', 'N', 2, bJ, n2, bJ, -1.0, w.W11, bJ, R + j0 + (j0 + bJ) * ldr, ldr, 1.0,
              Bnext, ell, cl.flag, 0));
      // re-sample: Omega' (A(rows > j0+bJ, trailing) - Y W^T)
      const int64_t mt = m - j0 - bJ;
      const int64_t kk = j0 + bJ;
      const int64_t* tcols = jpvt + j0 + bJ;
      CKL(1, rq::launch_gaussian(seed, kResampleStreamBase + J, ell, mt, w.omega, ell, cl.flag, cl.st));
      CK(gemm(cl, 'N', 'N', 0, ell, n2, mt, 1.0, w.omega, ell, dA + kk, lda, 0.0, Bnext, ell,
              cl.flag, 1, tcols));
      CK(gemm(cl, 'N', 'N', 0, ell, kk, mt, 1.0, w.omega, ell, Y + kk, ldy, 0.0, w.OY, ell, cl.flag,
              1));
      CK(gemm(cl, 'N', 'N', 0, ell, n2, kk, -1.0, w.OY, ell, w.Wt + kk * k, k, 1.0, Bnext, ell,
              cl.flag, 1));
    }
  }
  return RQRCP_OK;
}

}  // namespace

int trqrcp(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k, int b,
           int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, double* dY, int64_t ldy,
           double* dR, int64_t ldr) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (k < 1 || k > std::min(m, n)) return -6;
  if (b < 1) return -7;
  if (p < 0) return -8;
  if (!d_jpvt) return -10;
  if (!d_tau) return -11;
  if (!dY) return -12;
  if (ldy < m) return -13;
  if (!dR) return -14;
  if (ldr < k) return -15;
  if (b > k) b = (int)k;
  const int ell = b + p;
  if (!sizes_fit(h->num_sms, m, n, b, ell)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'T', m, n, k, b, p, &cl);
  if (r) return r;
  return trqrcp_core(cl, m, n, dA, lda, k, b, ell, seed, d_jpvt, d_tau, dY, ldy, dR, ldr);
}

// Arguments 1-8, shared by tuxv, tuxv_iter and tuxv_svd (same positions).
int check_tuxv_head(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda,
                    int64_t k, int b, int p) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (k < 1 || k > std::min(m, n)) return -6;
  if (b < 1) return -7;
  if (p < 0) return -8;
  return RQRCP_OK;
}

int check_tuxv_sizes(rqrcp_handle_t h, int64_t m, int64_t n, int64_t k, int b, int p) {
  if (b > k) b = (int)k;
  if (!sizes_fit(h->num_sms, m, n, b, b + p) || !rq::panel_fits(n, b, h->num_sms))
    return RQRCP_ERR_UNSUPPORTED;
  return RQRCP_OK;
}

int tuxv_core(Call& cl, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k, int b,
              int ell, uint64_t seed, int jmax, double* dU, int64_t ldu, double* dX, int64_t ldx,
              double* dV, int64_t ldv) {
  Work& w = cl.w;
  int r;
  // Alg. 7: TRQRCP, then Z0 = R P^T
  if ((r = trqrcp_core(cl, m, n, dA, lda, k, b, ell, seed, w.jpvt, w.tau, w.Yk, m, w.Rk, k))) return r;
  // Z0^T (n x k) into V's storage: V(jpvt[c], :) = R(:, c)^T
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_scatter_transpose(w.Rk, k, k, w.jpvt, n, dV, ldv, cl.st));
  }
  // LQ of Z0 as the QR of Z0^T; V1 = leading k columns of its Q
  if ((r = qr_core(cl, n, k, dV, ldv, b, w.tau2, w.Tall))) return r;
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_copy2d(dV, ldv, w.F, n, n, k, cl.st));
  }
  if ((r = orgqr_core(cl, n, k, w.F, n, b, w.Tall, dV, ldv))) return r;
  for (int j = 1;; j += 2) {
    // Alg. 7, odd j: Z = A V, then [U, X] = qr(Z) (X upper triangular)
    {
      PhaseScope ps(cl.h, PH_TRQ, 2.0 * (double)m * (double)n * (double)k);
      CK(gemm(cl, 'N', 'N', 0, m, k, n, 1.0, dA, lda, dV, ldv, 0.0, dU, ldu));
    }
    if ((r = qr_core(cl, m, k, dU, ldu, b, w.tau2, w.Tall))) return r;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      CKL(1, rq::launch_split_qr(dU, ldu, k, k, 0, nullptr, 0, dX, ldx, cl.st));
      CKL(1, rq::launch_copy2d(dU, ldu, w.F, m, m, k, cl.st));
    }
    if ((r = orgqr_core(cl, m, k, w.F, m, b, w.Tall, dU, ldu))) return r;
    if (j == jmax) break;
    // Alg. 7, even j: Z = U^T A, then [X, V^T] = lq(Z) through the QR of
    // Z^T = A^T U (X = R^T lower triangular)
    {
      PhaseScope ps(cl.h, PH_TRQ, 2.0 * (double)m * (double)n * (double)k);
      CK(gemm(cl, 'T', 'N', 0, n, k, m, 1.0, dA, lda, dU, ldu, 0.0, dV, ldv));
    }
    if ((r = qr_core(cl, n, k, dV, ldv, b, w.tau2, w.Tall))) return r;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      CKL(1, rq::launch_r_transposed(dV, ldv, k, dX, ldx, cl.st));
      CKL(1, rq::launch_copy2d(dV, ldv, w.F, n, n, k, cl.st));
    }
    if ((r = orgqr_core(cl, n, k, w.F, n, b, w.Tall, dV, ldv))) return r;
    if (j + 1 == jmax) break;
  }
  return RQRCP_OK;
}

int tuxv_iter(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k,
              int b, int p, uint64_t seed, int jmax, double* dU, int64_t ldu, double* dX,
              int64_t ldx, double* dV, int64_t ldv) {
  int r = check_tuxv_head(h, m, n, dA, lda, k, b, p);
  if (r) return r;
  if (jmax < 1) return -10;
  if (!dU) return -11;
  if (ldu < m) return -12;
  if (!dX) return -13;
  if (ldx < k) return -14;
  if (!dV) return -15;
  if (ldv < n) return -16;
  if ((r = check_tuxv_sizes(h, m, n, k, b, p))) return r;
  if (b > k) b = (int)k;
  Call cl;
  if ((r = begin(h, 'U', m, n, k, b, p, &cl))) return r;
  return tuxv_core(cl, m, n, dA, lda, k, b, b + p, seed, jmax, dU, ldu, dX, ldx, dV, ldv);
}

int tuxv_svd(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k,
             int b, int p, uint64_t seed, int jmax, double* dU, int64_t ldu, double* d_sigma,
             double* dV, int64_t ldv) {
  int r = check_tuxv_head(h, m, n, dA, lda, k, b, p);
  if (r) return r;
  if (jmax < 1) return -10;
  if (!dU) return -11;
  if (ldu < m) return -12;
  if (!d_sigma) return -13;
  if (!dV) return -14;
  if (ldv < n) return -15;
  if ((r = check_tuxv_sizes(h, m, n, k, b, p))) return r;
  if (b > k) b = (int)k;
  Call cl;
  if ((r = begin(h, 'U', m, n, k, b, p, &cl))) return r;
  Work& w = cl.w;
  const int64_t kk = k * k;
  double* X = w.svd;
  double* Ux = w.svd + 3 * kk;
  double* Vs = w.svd + 4 * kk;
  if ((r = tuxv_core(cl, m, n, dA, lda, k, b, b + p, seed, jmax, dU, ldu, X, k, dV, ldv)))
    return r;
  // X = Ux diag(sigma) Vs^T, then U <- U Ux and V <- V Vs
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    rq::JacobiArgs ja{X,  k,       (int)k,         w.svd + kk, w.svd + 2 * kk, Ux,
                      Vs, d_sigma, w.svd + 5 * kk, w.rotated,  cl.bar,         cl.status};
    CKL(1, rq::launch_jacobi_svd(ja, cl.h->num_sms, cl.st));
  }
  {
    PhaseScope ps(cl.h, PH_TRQ, 2.0 * (double)(m + n) * (double)k * (double)k);
    CK(gemm(cl, 'N', 'N', 0, m, k, k, 1.0, dU, ldu, Ux, k, 0.0, w.F, m));
    CKL(1, rq::launch_copy2d(w.F, m, dU, ldu, m, k, cl.st));
    CK(gemm(cl, 'N', 'N', 0, n, k, k, 1.0, dV, ldv, Vs, k, 0.0, w.F, n));
    CKL(1, rq::launch_copy2d(w.F, n, dV, ldv, n, k, cl.st));
  }
  return RQRCP_OK;
}

int tuxv(rqrcp_handle_t h, int64_t m, int64_t n, const double* dA, int64_t lda, int64_t k, int b,
         int p, uint64_t seed, double* dU, int64_t ldu, double* dX, int64_t ldx, double* dV,
         int64_t ldv) {
  int r = check_tuxv_head(h, m, n, dA, lda, k, b, p);
  if (r) return r;
  if (!dU) return -10;
  if (ldu < m) return -11;
  if (!dX) return -12;
  if (ldx < k) return -13;
  if (!dV) return -14;
  if (ldv < n) return -15;
  if ((r = check_tuxv_sizes(h, m, n, k, b, p))) return r;
  if (b > k) b = (int)k;
  Call cl;
  if ((r = begin(h, 'U', m, n, k, b, p, &cl))) return r;
  return tuxv_core(cl, m, n, dA, lda, k, b, b + p, seed, 1, dU, ldu, dX, ldx, dV, ldv);
}

int rqrcp_factor_mixed(rqrcp_handle_t h, int64_t m, int64_t n, float* dA, int64_t lda, int b,
                       int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, double* d_rdiag) {
  if (!h) return -1;
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (b < 1) return -6;
  if (p < 0) return -7;
  if (!d_jpvt) return -9;
  if (!d_tau) return -10;
  if (!d_rdiag) return -11;
  const int64_t k = std::min(m, n);
  if (b > k) b = (int)k;
  const int ell = b + p;
  if (!sizes_fit(h->num_sms, m, n, b, ell)) return RQRCP_ERR_UNSUPPORTED;
  Call cl;
  int r = begin(h, 'M', m, n, k, b, p, &cl);
  if (r) return r;
  Work& w = cl.w;
  {
    // Omega in FP64 from Philox, rounded for the BF16 sketch B = Omega A
    PhaseScope ps(cl.h, PH_SKETCH, 2.0 * ell * (double)m * (double)n);
    CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, w.omega, ell, nullptr, cl.st));
    CKL(1, rq::launch_convert_f64_f32(w.omega, ell, w.omega32, ell, ell, m, cl.st));
    CK(tcgemm(cl, 'N', 'N', ell, n, m, 1.0f, w.omega32, ell, dA, lda, 0.0f, w.B32, ell, 1));
    CKL(1, rq::launch_convert_f32_f64(w.B32, ell, w.B, ell, ell, n, cl.st));
    CKL(1, rq::launch_iota(d_jpvt, n, cl.st));
  }
  for (int64_t j0 = 0; j0 < k; j0 += b) {
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    const int64_t nc = n - j0, n2 = nc - bJ, mJ = m - j0;
    double* Bblk = w.B + j0 * ell;
    if ((r = sample_step(cl, Bblk, ell, nc, bJ, 1))) return r;
    {
      PhaseScope ps(cl.h, PH_PERM, 0.0);
      CKL(3, rq::launch_apply_swaps_f32(dA, lda, m, j0, w.swaps, bJ, d_jpvt, w.map, w.permbuf32,
                                        cl.st));
    }
    // FP64 panel, T and R diagonal; FP32 copies back into A and Y32
    float* P = dA + j0 + j0 * lda;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      CKL(1, rq::launch_convert_f32_f64(P, lda, w.P64, m, mJ, bJ, cl.st));
    }
    if ((r = panel_step(cl, w.P64, m, mJ, bJ, d_tau + j0, w.T, 1))) return r;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      CKL(1, rq::launch_panel_writeback(w.P64, m, mJ, bJ, P, lda, w.Y32, m, d_rdiag + j0, cl.st));
    }
    float* A2 = dA + j0 + (j0 + bJ) * lda;
    if (n2 > 0) {
      // trailing update with split-BF16 x3 tensor-core products
      PhaseScope ps(cl.h, PH_TRAIL, 4.0 * (double)mJ * (double)n2 * bJ + 2.0 * bJ * bJ * (double)n2);
      CKL(1, rq::launch_convert_f64_f32(w.T, bJ, w.T32, bJ, bJ, bJ, cl.st));
      CK(tcgemm(cl, 'T', 'N', bJ, n2, mJ, 1.0f, w.Y32, m, A2, lda, 0.0f, w.Z32, bJ, 3));
      CK(tcgemm(cl, 'T', 'N', bJ, n2, bJ, 1.0f, w.T32, bJ, w.Z32, bJ, 0.0f, w.W32, bJ, 3));
      CK(tcgemm(cl, 'N', 'N', mJ, n2, bJ, -1.0f, w.Y32, m, w.W32, bJ, 1.0f, A2, lda, 3));
    }
    if (j0 + bJ < k) {
      // Eq. (3) with R11 from the FP64 panel and R12 widened from FP32, the
      // product FP64-accurate on the tensor cores (the split-BF16 slice
      // buffers are free here); an exactly singular R11 keeps S12 (no
      // re-sample in this mode)
      PhaseScope ps(cl.h, PH_SUPD, (double)bJ * bJ * bJ / 3.0 + 2.0 * bJ * bJ * (double)n2);
      CKL(1, rq::launch_w11(Bblk, ell, w.P64, m, bJ, w.W11, cl.flag, cl.status, cl.st));
      CKL(1, rq::launch_convert_f32_f64(A2, lda, w.R12, bJ, bJ, n2, cl.st));
      if ((r = sample_update_product(cl, w.W11, bJ, w.R12, bJ, n2, Bblk + (int64_t)bJ * ell, ell,
                                     w.tslA, w.tslcapA, w.exB, w.tslB, w.tslcapB, w.exA)))
        return r;
    }
  }
  return RQRCP_OK;
}

}  // extern "C"

namespace {

// Argument checks of trqrcp_mixed (0, -i for argument i, or
// RQRCP_ERR_UNSUPPORTED); b is clamped to k.
int check_trqrcp_mixed(int num_sms, int64_t m, int64_t n, const float* dA, int64_t lda, int64_t k,
                       int& b, int p, const int64_t* d_jpvt, const double* d_tau, const float* dY,
                       int64_t ldy, const float* dR, int64_t ldr, const double* d_rdiag) {
  if (m < 1) return -2;
  if (n < 1) return -3;
  if (!dA) return -4;
  if (lda < m) return -5;
  if (k < 1 || k > std::min(m, n)) return -6;
  if (b < 1) return -7;
  if (p < 0) return -8;
  if (!d_jpvt) return -10;
  if (!d_tau) return -11;
  if (!dY) return -12;
  if (ldy < m) return -13;
  if (!dR) return -14;
  if (ldr < k) return -15;
  if (!d_rdiag) return -16;
  if (b > k) b = (int)k;
  if (!sizes_fit(num_sms, m, n, b, b + p)) return RQRCP_ERR_UNSUPPORTED;
  return RQRCP_OK;
}

// Alg. 6 in mixed precision on the call's stream and scratch (arguments
// already checked, b <= k).
int trqrcp_mixed_run(Call& cl, int64_t m, int64_t n, const float* dA, int64_t lda, int64_t k,
                     int b, int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, float* dY,
                     int64_t ldy, float* dR, int64_t ldr, double* d_rdiag) {
  const int ell = b + p;
  int r = RQRCP_OK;
  Work& w = cl.w;
  float* Ahat = w.Y32;
  float* Wt = w.W32;                                   // k x n, ld k
  float* YY = reinterpret_cast<float*>(w.Wt);          // b x k, ld b
  {
    PhaseScope ps(cl.h, PH_SKETCH, 2.0 * ell * (double)m * (double)n);
    CKL(1, rq::launch_gaussian(seed, kOmegaStream, ell, m, w.omega, ell, nullptr, cl.st));
    CKL(1, rq::launch_convert_f64_f32(w.omega, ell, w.omega32, ell, ell, m, cl.st));
    CK(tcgemm(cl, 'N', 'N', ell, n, m, 1.0f, w.omega32, ell, dA, lda, 0.0f, w.B32, ell, 1));
    CKL(1, rq::launch_convert_f32_f64(w.B32, ell, w.B, ell, ell, n, cl.st));
  }
  {
    PhaseScope ps(cl.h, PH_OTHER, 0.0);
    CKL(1, rq::launch_iota(d_jpvt, n, cl.st));
    CK(cudaMemset2DAsync(dY, ldy * sizeof(float), 0, m * sizeof(float), k, cl.st));
    CK(cudaMemset2DAsync(dR, ldr * sizeof(float), 0, k * sizeof(float), n, cl.st));
    CK(cudaMemsetAsync(Wt, 0, sizeof(float) * k * n, cl.st));
  }
  for (int64_t j0 = 0; j0 < k; j0 += b) {
    const int bJ = (int)std::min<int64_t>(b, k - j0);
    const int64_t nc = n - j0, n2 = nc - bJ, mJ = m - j0;
    double* Bblk = w.B + j0 * ell;
    if ((r = sample_step(cl, Bblk, ell, nc, bJ, 1))) return r;
    {
      PhaseScope ps(cl.h, PH_PERM, 0.0);
      CKL(3, rq::launch_apply_swaps_f32(Wt, k, j0, j0, w.swaps, bJ, d_jpvt, w.map, w.permbuf32, cl.st));
      CKL(3, rq::launch_apply_swaps_f32(dR, ldr, j0, j0, w.swaps, bJ, nullptr, w.map, w.permbuf32,
                                        cl.st));
    }
    {
      // selected columns A_hat = A(:, sel) - Y1 W1^T(:, sel) on rows j0..m-1
      PhaseScope ps(cl.h, PH_TRQ, 2.0 * (double)mJ * bJ * (double)j0);
      CKL(1, rq::launch_gather_cols_f32(dA, lda, j0, mJ, d_jpvt + j0, bJ, Ahat, m, cl.st));
      if (j0 > 0)
        CK(tcgemm(cl, 'N', 'N', mJ, bJ, j0, -1.0f, dY + j0, ldy, Wt + j0 * k, k, 1.0f, Ahat, m, 3));
      CKL(1, rq::launch_convert_f32_f64(Ahat, m, w.P64, m, mJ, bJ, cl.st));
    }
    if ((r = panel_step(cl, w.P64, m, mJ, bJ, d_tau + j0, w.T, 1))) return r;
    {
      PhaseScope ps(cl.h, PH_OTHER, 0.0);
      // Y (explicit, FP32) and R11 (FP32, diagonal also in FP64)
      CKL(1, rq::launch_panel_writeback(w.P64, m, mJ, bJ, Ahat, m, dY + j0 + j0 * ldy, ldy,
                                        d_rdiag + j0, cl.st));
      CKL(1, rq::launch_copy_upper_f32(Ahat, m, bJ, dR + j0 + j0 * ldr, ldr, cl.st));
      CKL(1, rq::launch_convert_f64_f32(w.T, bJ, w.T32, bJ, bJ, bJ, cl.st));
    }
    if (n2 > 0) {
      PhaseScope ps(cl.h, PH_TRQ,
                    2.0 * bJ * (double)mJ * (double)n2 + 2.0 * bJ * (double)mJ * j0 +
                        2.0 * bJ * (double)j0 * (double)n2 + 2.0 * bJ * bJ * (double)n2 +
                        2.0 * bJ * (double)(j0 + bJ) * (double)n2);
      const int64_t* tcols = d_jpvt + j0 + bJ;
      const float* Y2 = dY + j0 + j0 * ldy;
      // W2^T = T2^T (Y2^T A(:, trailing) - (Y2^T Y1) W1^T(:, trailing))
      CK(tcgemm(cl, 'T', 'N', bJ, n2, mJ, 1.0f, Y2, ldy, dA + j0, lda, 0.0f, w.Z32, bJ, 3, tcols));
      if (j0 > 0) {
        CK(tcgemm(cl, 'T', 'N', bJ, j0, mJ, 1.0f, Y2, ldy, dY + j0, ldy, 0.0f, YY, bJ, 3));
        CK(tcgemm(cl, 'N', 'N', bJ, n2, j0, -1.0f, YY, bJ, Wt + (j0 + bJ) * k, k, 1.0f, w.Z32, bJ,
                  3));
      }
      CK(tcgemm(cl, 'T', 'N', bJ, n2, bJ, 1.0f, w.T32, bJ, w.Z32, bJ, 0.0f, Wt + j0 + (j0 + bJ) * k,
                k, 3));
      // new rows of R: A(rows J, trailing) - Y(rows J, :) W^T(:, trailing)
      float* Rrows = dR + j0 + (j0 + bJ) * ldr;
      CKL(1, rq::launch_gather_cols_f32(dA, lda, j0, bJ, tcols, n2, Rrows, ldr, cl.st));
      CK(tcgemm(cl, 'N', 'N', bJ, n2, j0 + bJ, -1.0f, dY + j0, ldy, Wt + (j0 + bJ) * k, k, 1.0f,
                Rrows, ldr, 3));
    }
    if (j0 + bJ < k) {
      PhaseScope ps(cl.h, PH_SUPD, (double)bJ * bJ * bJ / 3.0 + 2.0 * bJ * bJ * (double)n2);
      CKL(1, rq::launch_w11(Bblk, ell, w.P64, m, bJ, w.W11, cl.flag, cl.status, cl.st));
      CKL(1, rq::launch_convert_f32_f64(dR + j0 + (j0 + bJ) * ldr, ldr, w.R12, bJ, bJ, n2, cl.st));
      if ((r = sample_update_product(cl, w.W11, bJ, w.R12, bJ, n2, Bblk + (int64_t)bJ * ell, ell,
                                     w.tslA, w.tslcapA, w.exB, w.tslB, w.tslcapB, w.exA)))
        return r;
    }
  }
  return RQRCP_OK;
}


}  // namespace

extern "C" {

int trqrcp_mixed(rqrcp_handle_t h, int64_t m, int64_t n, const float* dA, int64_t lda, int64_t k,
                 int b, int p, uint64_t seed, int64_t* d_jpvt, double* d_tau, float* dY,
                 int64_t ldy, float* dR, int64_t ldr, double* d_rdiag) {
  if (!h) return -1;
  int r = check_trqrcp_mixed(h->num_sms, m, n, dA, lda, k, b, p, d_jpvt, d_tau, dY, ldy, dR, ldr,
                             d_rdiag);
  if (r) return r;
  Call cl;
  r = begin(h, 'V', m, n, k, b, p, &cl);
  if (r) return r;
  return trqrcp_mixed_run(cl, m, n, dA, lda, k, b, p, seed, d_jpvt, d_tau, dY, ldy, dR, ldr,
                          d_rdiag);
}

// ---------------------------------------------------------------- batched
namespace {

// device control words of the persistent kernel: claim counter (8 bytes),
// exit counter (4 bytes), then one grid barrier per team
constexpr size_t kCtlBarOffset = 64;
constexpr int kMaxTeams = 512;
// per team 8 phase times (ns) of the instrumentation, after the barriers
constexpr size_t kCtlTraceOffset = kCtlBarOffset + sizeof(rq::GridBarrier) * kMaxTeams;
constexpr size_t kCtlBytes = kCtlTraceOffset + sizeof(long long) * 8 * kMaxTeams;
constexpr int kTableReserve = 1024;

int max_teams(rqrcp_handle_t h) { return std::max(1, h->num_sms / h->bt_G); }

bool same_limits(const rq::BatchLimits& a, const rq::BatchLimits& b) {
  return a.m == b.m && a.n == b.n && a.k == b.k && a.b == b.b && a.ell == b.ell;
}

// Scratch of `teams` teams for problems up to `want` (grown, never shrunk).
int ensure_batch(rqrcp_handle_t h, const rq::BatchLimits& want, int teams) {
  rq::BatchLimits lim = h->bt_lim;
  lim.m = std::max(lim.m, want.m);
  lim.n = std::max(lim.n, want.n);
  lim.k = std::max(lim.k, want.k);
  lim.b = std::max(lim.b, want.b);
  lim.ell = std::max(lim.ell, want.ell);
  const int nt = std::max(teams, h->bt_teams);
  if (h->bt_ctl && h->bt_scratch && same_limits(lim, h->bt_lim) && nt == h->bt_teams)
    return RQRCP_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  rq::BatchLayout L{};
  const size_t tb = rq::batch_team_bytes(lim, h->bt_G, &L);
  if (e == cudaSuccess && h->bt_scratch) e = cudaFree(h->bt_scratch);
  h->bt_scratch = nullptr;
  h->bt_teams = 0;
  if (e == cudaSuccess) e = cudaMalloc(&h->bt_scratch, tb * nt);
  if (e == cudaSuccess && !h->bt_ctl) e = cudaMalloc(&h->bt_ctl, kCtlBytes);
  if (e != cudaSuccess) {
    if (h->bt_scratch) cudaFree(h->bt_scratch);
    h->bt_scratch = nullptr;
    h->err = std::string("batched scratch: ") + cudaGetErrorString(e);
    return RQRCP_ERR_ALLOC;
  }
  h->bt_lim = lim;
  h->bt_L = L;
  h->bt_team_bytes = tb;
  h->bt_teams = nt;
  return RQRCP_OK;
}

// Device table and its page-locked staging for `nprob` descriptors.
int ensure_table(rqrcp_handle_t h, int nprob) {
  if (h->bt_cap >= nprob && h->bt_table && h->bt_stage) return RQRCP_OK;
  const int cap = std::max(nprob, std::max(kTableReserve, 2 * h->bt_cap));
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (h->bt_table) cudaFree(h->bt_table);
  if (h->bt_stage) cudaFreeHost(h->bt_stage);
  h->bt_table = nullptr;
  h->bt_stage = nullptr;
  h->bt_cap = 0;
  if (e == cudaSuccess) e = cudaMalloc(&h->bt_table, sizeof(rqrcp_problem) * cap);
  if (e == cudaSuccess) e = cudaHostAlloc(&h->bt_stage, sizeof(rqrcp_problem) * cap, 0);
  if (e != cudaSuccess) {
    h->err = std::string("batched table: ") + cudaGetErrorString(e);
    return RQRCP_ERR_ALLOC;
  }
  h->bt_cap = cap;
  return RQRCP_OK;
}

// Argument checks of one problem (0, -i for field i in the argument order of
// trqrcp_mixed, or RQRCP_ERR_UNSUPPORTED); b is clamped to k.
int check_problem(const rqrcp_handle_t h, rqrcp_problem& q) {
  if (q.m < 1) return -2;
  if (q.n < 1) return -3;
  if (!q.dA) return -4;
  if (q.lda < q.m) return -5;
  if (q.k < 1 || q.k > std::min(q.m, q.n)) return -6;
  if (q.b < 1) return -7;
  if (q.p < 0) return -8;
  if (!q.d_jpvt) return -10;
  if (!q.d_tau) return -11;
  if (!q.dY) return -12;
  if (q.ldy < q.m) return -13;
  if (!q.dR) return -14;
  if (q.ldr < q.k) return -15;
  if (!q.d_rdiag) return -16;
  if (q.b > q.k) q.b = (int)q.k;
  if (q.b > kMaxB || q.b + q.p > kMaxEll) return RQRCP_ERR_UNSUPPORTED;
  if (!rq::batch_fits(q.m, q.n, q.b, q.b + q.p, h->bt_G)) return RQRCP_ERR_UNSUPPORTED;
  return RQRCP_OK;
}

double problem_flops(const rqrcp_problem& q) {
  return 2.0 * q.m * q.n * q.k + 2.0 * (q.b + q.p) * (double)q.m * q.n;
}

rq::BatchLaunch batch_launch(rqrcp_handle_t h, int teams) {
  rq::BatchLaunch bl{};
  bl.next = reinterpret_cast<unsigned long long*>(h->bt_ctl);
  bl.exited = reinterpret_cast<int*>(h->bt_ctl + 8);
  bl.G = h->bt_G;
  bl.teams = teams;
  bl.scratch = h->bt_scratch;
  bl.team_bytes = h->bt_team_bytes;
  bl.L = h->bt_L;
  bl.bars = reinterpret_cast<rq::GridBarrier*>(h->bt_ctl + kCtlBarOffset);
  bl.status = h->state;
  bl.trace = h->prof ? reinterpret_cast<long long*>(h->bt_ctl + kCtlTraceOffset) : nullptr;
  return bl;
}

// Clears the phase timers of the batched kernel when profiling was (re)enabled.
cudaError_t batch_trace_prepare(rqrcp_handle_t h) {
  if (!h->prof || !h->bt_trace_clear || !h->bt_ctl) return cudaSuccess;
  h->bt_trace_clear = false;
  return cudaMemsetAsync(h->bt_ctl + kCtlTraceOffset, 0, sizeof(long long) * 8 * kMaxTeams,
                         h->stream);
}

}  // namespace

int rqrcp_reserve_batched(rqrcp_handle_t h, int teams, int64_t m, int64_t n, int64_t k, int b,
                          int p) {
  if (!h) return -1;
  if (teams < 0) return -2;
  if (m < 1 || n < 1 || k < 1 || k > std::min(m, n) || b < 1 || p < 0) return -3;
  if (b > k) b = (int)k;
  if (b > kMaxB || b + p > kMaxEll || !rq::batch_fits(m, n, b, b + p, h->bt_G))
    return RQRCP_ERR_UNSUPPORTED;
  const int nt = teams == 0 ? max_teams(h) : std::min(teams, max_teams(h));
  int r = ensure_batch(h, rq::BatchLimits{m, n, k, b, b + p}, nt);
  if (r) return r;
  return ensure_table(h, kTableReserve);
}

int trqrcp_batched(rqrcp_handle_t h, int nprob, const rqrcp_problem* probs, int teams) {
  if (!h) return -1;
  if (nprob < 0) return -2;
  if (nprob > 0 && !probs) return -3;
  if (teams < 0) return -4;
  if (nprob == 0) return RQRCP_OK;
  // every problem is checked before anything is enqueued
  std::vector<rqrcp_problem> qs(probs, probs + nprob);
  rq::BatchLimits lim{1, 1, 1, 1, 1};
  for (int i = 0; i < nprob; ++i) {
    const int r = check_problem(h, qs[i]);
    if (r) {
      h->err = "trqrcp_batched: problem " + std::to_string(i) + ": status " + std::to_string(r);
      return RQRCP_ERR_BATCH;
    }
    lim.m = std::max(lim.m, qs[i].m);
    lim.n = std::max(lim.n, qs[i].n);
    lim.k = std::max(lim.k, qs[i].k);
    lim.b = std::max(lim.b, qs[i].b);
    lim.ell = std::max(lim.ell, qs[i].b + qs[i].p);
  }
  int nt = teams == 0 ? max_teams(h) : std::min(teams, max_teams(h));
  nt = std::min(nt, nprob);
  int r = ensure_batch(h, lim, nt);
  if (r) return r;
  if ((r = ensure_table(h, nprob))) return r;
  // longest first, by algorithmic flops: the teams claim the table in order
  std::stable_sort(qs.begin(), qs.end(), [](const rqrcp_problem& a, const rqrcp_problem& c) {
    return problem_flops(a) > problem_flops(c);
  });
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
  // the staging buffer may still feed the copy of the previous batch: wait
  // for that copy (not for the whole stream)
  if (cs == cudaStreamCaptureStatusNone && h->bt_copy_pending) {
    cudaError_t e = cudaEventSynchronize(h->bt_copy_ev);
    if (e != cudaSuccess) {
      h->err = std::string("trqrcp_batched: ") + cudaGetErrorString(e);
      return RQRCP_ERR_CUDA;
    }
    h->bt_copy_pending = false;
  }
  std::copy(qs.begin(), qs.end(), h->bt_stage);
  double fl = 0.0;
  for (const auto& q : qs) fl += problem_flops(q);
  PhaseScope ps(h, PH_TRQ, fl);
  cudaError_t e = batch_trace_prepare(h);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->bt_table, h->bt_stage, sizeof(rqrcp_problem) * nprob,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
    if (!h->bt_copy_ev) e = cudaEventCreateWithFlags(&h->bt_copy_ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(h->bt_copy_ev, h->stream);
    if (e == cudaSuccess) h->bt_copy_pending = true;
  }
  rq::BatchLaunch bl = batch_launch(h, nt);
  bl.table = h->bt_table;
  bl.nprob = nprob;
  if (e == cudaSuccess) e = rq::launch_batch_trqrcp(bl, h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("trqrcp_batched: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  count_launch(h, 1);
  return RQRCP_OK;
}

// ---------------------------------------------------------------- serving ring
namespace {

constexpr unsigned int kServerIdlePolls = 200000;  // ~0.2-0.5 s of an empty ring

rq::RequestRing* ring_host(rqrcp_handle_t h) {
  return reinterpret_cast<rq::RequestRing*>(h->ring_host);
}
rqrcp_problem* ring_slots(char* base) {
  return reinterpret_cast<rqrcp_problem*>(base + sizeof(rq::RequestRing));
}
volatile int* ring_info(char* base, int cap) {
  return reinterpret_cast<volatile int*>(ring_slots(base) + cap);
}
volatile long long* ring_done(char* base, int cap) {
  return reinterpret_cast<volatile long long*>(ring_info(base, cap) + ((cap + 1) & ~1));
}

// (Re)launches the persistent kernel on the ring; tickets continue from the
// device claim counter when `keep` is set.
int server_launch(rqrcp_handle_t h, bool keep) {
  rq::RequestRing* r = ring_host(h);
  r->running = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  rq::BatchLaunch bl = batch_launch(h, h->bt_server_teams);
  bl.ring = h->ring_dev;
  bl.idle_polls = kServerIdlePolls;
  bl.keep_next = keep ? 1 : 0;
  bl.trace = nullptr;
  cudaError_t e = rq::launch_batch_trqrcp(bl, h->stream);
  if (e != cudaSuccess) {
    r->running = 0;
    h->err = std::string("server launch: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  count_launch(h, 1);
  h->ring_running = true;
  return RQRCP_OK;
}

}  // namespace

int rqrcp_server_start(rqrcp_handle_t h, int capacity, int teams, int64_t m, int64_t n,
                       int64_t k, int b, int p) {
  if (!h) return -1;
  if (capacity < 1 || capacity > (1 << 20)) return -2;
  if (teams < 0) return -3;
  if (h->ring_running) {
    h->err = "server_start: a server is already running on this handle";
    return RQRCP_ERR_UNSUPPORTED;
  }
  int r = rqrcp_reserve_batched(h, teams, m, n, k, b, p);
  if (r) return r;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess && h->ring_cap != capacity) {
    if (h->ring_host) cudaFreeHost(h->ring_host);
    h->ring_host = nullptr;
    h->ring_cap = 0;
    e = cudaHostAlloc(&h->ring_host, rq::request_ring_bytes(capacity),
                      cudaHostAllocMapped | cudaHostAllocPortable);
    if (e == cudaSuccess) h->ring_cap = capacity;
  }
  void* dptr = nullptr;
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dptr, h->ring_host, 0);
  if (e != cudaSuccess) {
    h->err = std::string("server_start: ") + cudaGetErrorString(e);
    return RQRCP_ERR_ALLOC;
  }
  std::memset(h->ring_host, 0, rq::request_ring_bytes(capacity));
  rq::RequestRing* rg = ring_host(h);
  rg->cap = capacity;
  h->ring_dev = static_cast<rq::RequestRing*>(dptr);
  h->ring_tail = 0;
  h->bt_server_teams = teams == 0 ? h->bt_teams : std::min(teams, h->bt_teams);
  return server_launch(h, false);
}

int rqrcp_server_submit(rqrcp_handle_t h, const rqrcp_problem* prob, int64_t* ticket) {
  if (!h) return -1;
  if (!prob) return -2;
  if (!ticket) return -3;
  if (!h->ring_running || !h->ring_host) {
    h->err = "server_submit: no server running (rqrcp_server_start)";
    return RQRCP_ERR_UNSUPPORTED;
  }
  rqrcp_problem q = *prob;
  int r = check_problem(h, q);
  if (r) return r < 0 ? -2 : r;
  if (q.m > h->bt_lim.m || q.n > h->bt_lim.n || q.k > h->bt_lim.k || q.b > h->bt_lim.b ||
      q.b + q.p > h->bt_lim.ell) {
    h->err = "server_submit: problem larger than the sizes the server was started for";
    return RQRCP_ERR_UNSUPPORTED;
  }
  rq::RequestRing* rg = ring_host(h);
  const int cap = h->ring_cap;
  const int64_t t = h->ring_tail;
  const int slot = (int)(t % cap);
  // the slot is free once the request that used it last is finished
  if (t >= cap && ring_done(h->ring_host, cap)[slot] != (long long)(t - cap + 1)) return RQRCP_ERR_BUSY;
  ring_slots(h->ring_host)[slot] = q;
  ring_info(h->ring_host, cap)[slot] = 0;
  std::atomic_thread_fence(std::memory_order_release);
  reinterpret_cast<volatile long long*>(&rg->tail)[0] = (long long)(t + 1);
  std::atomic_thread_fence(std::memory_order_seq_cst);
  h->ring_tail = t + 1;
  *ticket = t;
  // every team may have left on an idle ring: start the kernel again
  if (reinterpret_cast<volatile int*>(&rg->running)[0] == 0) {
    r = server_launch(h, true);
    if (r) return r;
  }
  return RQRCP_OK;
}

int rqrcp_server_poll(rqrcp_handle_t h, int64_t ticket, int* info) {
  if (!h) return -1;
  if (!h->ring_host || ticket < 0 || ticket >= h->ring_tail) return -2;
  const int cap = h->ring_cap;
  const int slot = (int)(ticket % cap);
  const long long d = ring_done(h->ring_host, cap)[slot];
  std::atomic_thread_fence(std::memory_order_acquire);
  if (d == (long long)ticket + 1) {
    if (info) *info = ring_info(h->ring_host, cap)[slot];
    return 1;
  }
  if (d > (long long)ticket + 1) return -2;  // the slot has been reused since
  rq::RequestRing* rg = ring_host(h);
  if (h->ring_running && reinterpret_cast<volatile int*>(&rg->running)[0] == 0 &&
      reinterpret_cast<volatile int*>(&rg->stop)[0] == 0) {
    // the teams left while this request was being published: relaunch
    const int r = server_launch(h, true);
    if (r) return r;
  }
  return 0;
}

int rqrcp_server_stop(rqrcp_handle_t h) {
  if (!h) return -1;
  if (!h->ring_host || !h->ring_running) return RQRCP_OK;
  rq::RequestRing* rg = ring_host(h);
  reinterpret_cast<volatile int*>(&rg->stop)[0] = 1;
  std::atomic_thread_fence(std::memory_order_seq_cst);
  h->ring_running = false;
  return RQRCP_OK;
}

int rqrcp_gemm_bf16x(rqrcp_handle_t h, char transA, char transB, int64_t m, int64_t n, int64_t k,
                     float alpha, const float* dA, int64_t lda, const float* dB, int64_t ldb,
                     float beta, float* dC, int64_t ldc, int slices) {
  if (!h) return -1;
  if (transA != 'N' && transA != 'T') return -2;
  if (transB != 'N' && transB != 'T') return -3;
  if (m < 0) return -4;
  if (n < 0) return -5;
  if (k < 0) return -6;
  const int64_t arows = transA == 'N' ? m : k, brows = transB == 'N' ? k : n;
  if (!dA && m * k > 0) return -8;
  if (lda < std::max<int64_t>(1, arows)) return -9;
  if (!dB && n * k > 0) return -10;
  if (ldb < std::max<int64_t>(1, brows)) return -11;
  if (!dC && m * n > 0) return -13;
  if (ldc < std::max<int64_t>(1, m)) return -14;
  if (slices != 1 && slices != 3) return -15;
  if (m == 0 || n == 0) return RQRCP_OK;
  Call cl;
  int r = begin(h, 'G', m, n, k, 1, 0, &cl);
  if (r) return r;
  PhaseScope ps(h, PH_TRAIL, 2.0 * (double)m * (double)n * (double)k);
  CK(tcgemm(cl, transA, transB, m, n, k, alpha, dA, lda, dB, ldb, beta, dC, ldc, slices));
  return RQRCP_OK;
}

int rqrcp_gemm_f64x(rqrcp_handle_t h, char transA, char transB, int64_t m, int64_t n, int64_t k,
                    double alpha, const double* dA, int64_t lda, const double* dB, int64_t ldb,
                    double beta, double* dC, int64_t ldc) {
  if (!h) return -1;
  if (transA != 'N' && transA != 'T') return -2;
  if (transB != 'N' && transB != 'T') return -3;
  if (m < 0) return -4;
  if (n < 0) return -5;
  if (k < 0) return -6;
  const int64_t arows = transA == 'N' ? m : k, brows = transB == 'N' ? k : n;
  if (!dA && m * k > 0) return -8;
  if (lda < std::max<int64_t>(1, arows)) return -9;
  if (!dB && n * k > 0) return -10;
  if (ldb < std::max<int64_t>(1, brows)) return -11;
  if (!dC && m * n > 0) return -13;
  if (ldc < std::max<int64_t>(1, m)) return -14;
  if (m == 0 || n == 0) return RQRCP_OK;
  Call cl;
  int r = begin(h, 'X', m, n, std::max<int64_t>(k, 1), 1, 0, &cl);
  if (r) return r;
  PhaseScope ps(h, PH_TRAIL, 2.0 * (double)m * (double)n * (double)k);
  // rows of op(A): stored columns when transposed; columns of op(B): stored
  // columns when not transposed
  CKL(rq::oz_slice_launches(transA == 'T', k),
      rq::launch_oz_slice(dA, lda, transA == 'T', 0, m, k, cl.w.slA, cl.w.exA, cl.st));
  CKL(rq::oz_slice_launches(transB == 'N', k),
      rq::launch_oz_slice(dB, ldb, transB == 'N', 0, n, k, cl.w.slB, cl.w.exB, cl.st));
  float* part = reinterpret_cast<float*>(cl.w.skpart);
  const size_t pcap = 2 * cl.w.skcap;
  rq::OzGemmArgs g{m,  n,   rq::oz_kpad(k), cl.w.slA, cl.w.exA, cl.w.slB,     cl.w.exB, alpha,
                   beta, dC, ldc,           cl.status, part,    pcap,         cl.h->num_sms};
  CKL(rq::oz_launches(m, n, g.Kp, cl.h->num_sms, pcap), rq::launch_oz_gemm(g, cl.st));
  return RQRCP_OK;
}

int rqrcp_profile(rqrcp_handle_t h, int enable) {
  if (!h) return -1;
  if (enable) {
    h->ev_used = 0;
    for (int i = 0; i < RQRCP_NPHASE; ++i) {
      h->flops[i] = 0.0;
      h->launches[i] = 0;
    }
    h->bt_trace_clear = true;
  }
  h->prof = enable != 0;
  return RQRCP_OK;
}

int rqrcp_profile_read(rqrcp_handle_t h, int nphase, double* ms, double* flops, int64_t* launches) {
  if (!h) return -1;
  if (nphase < 0 || nphase > RQRCP_NPHASE) return -2;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    h->err = std::string("profile_read: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  double acc[RQRCP_NPHASE] = {};
  for (size_t i = 0; i < h->ev_used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, h->events[2 * i], h->events[2 * i + 1]) == cudaSuccess)
      acc[h->ev_phase[i]] += t;
  }
  for (int i = 0; i < nphase; ++i) {
    if (ms) ms[i] = acc[i];
    if (flops) flops[i] = h->flops[i];
    if (launches) launches[i] = h->launches[i];
  }
  return RQRCP_OK;
}

int rqrcp_batched_profile(rqrcp_handle_t h, int nphase, double* team_ms) {
  if (!h) return -1;
  if (nphase < 0 || nphase > RQRCP_NPHASE) return -2;
  if (!team_ms && nphase > 0) return -3;
  for (int i = 0; i < nphase; ++i) team_ms[i] = 0.0;
  if (!h->bt_ctl || h->bt_teams == 0) return RQRCP_OK;
  std::vector<long long> t((size_t)8 * h->bt_teams);
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.data(), h->bt_ctl + kCtlTraceOffset, sizeof(long long) * t.size(),
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    h->err = std::string("batched_profile: ") + cudaGetErrorString(e);
    return RQRCP_ERR_CUDA;
  }
  for (int tm = 0; tm < h->bt_teams; ++tm)
    for (int i = 0; i < nphase; ++i) team_ms[i] += 1e-6 * (double)t[(size_t)8 * tm + i];
  return RQRCP_OK;
}

}  // extern "C"
