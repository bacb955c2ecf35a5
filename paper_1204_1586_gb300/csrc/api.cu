// C ABI of cpgrad: argument checks, planning, workspace layout and the launch
// sequences of Algorithm 2 (all-mode gradient), Section 3.2 (single-mode
// gradient) and Section 4 (fast CP_ALS).
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "als.cuh"
#include "als_df.cuh"
#include "chain.cuh"
#include "common.cuh"
#include "consumers.cuh"
#include "lead_dispatch.cuh"
#include "tensor_map.h"
#include "api_internal.h"
#include "lead_tc_dispatch.cuh"
#include "lead_ws.cuh"

using namespace cpg;

namespace {

thread_local uint64_t g_launches = 0;

// Optional timing of launches: CUDA events recorded on the launch stream
// around every leading-contraction kernel (mode 1) or every kernel (mode 2)
// while enabled; each record keeps the launch's kind (cpgrad.h).
struct LeadTiming {
  bool on = false;
  bool all = false;
  int n = 0;
  static constexpr int kMax = 4096;
  cudaEvent_t ev[2 * kMax] = {};
  int sides[kMax] = {};
  bool made = false;
};
LeadTiming g_timing;

// Kinds of timed launches: 1-3 leading passes (sides), 10+ the rest.
enum LaunchKind : int {
  kKindChain = 10,   // finishing contraction or recursion (segmented dot)
  kKindMode = 11,    // fused ALS mode: G, then the update (FP32 data)
  kKindGram = 12,    // Gram matrices of all factors
  kKindKron = 13,    // Kronecker vector of a run of modes
  kKindNorm = 14,    // ||Y||^2 from partial sums
  kKindUpdate = 15,  // ALS update (FP64 data), multiplicative update (eq. 2.18)
  kKindModelTerm = 16,  // model term of the cost gradient (eq. 2.13) and first-order step (eq. 2.15)
  kKindRows = 17,       // Khatri-Rao rows of a CUDA-core leading pass, built once per pass
  kKindPitch = 18       // copy of Y_(1:k) with a 16-byte column pitch
};

// Records a start event at construction and an end event at destruction when
// timing is on for this kind of launch.
class Timed {
 public:
  Timed(cudaStream_t st, int kind) : st_(st), kind_(kind) {
    if (g_timing.on && g_timing.made && g_timing.n < LeadTiming::kMax && (kind < kKindChain || g_timing.all)) {
      slot_ = g_timing.n++;
      cudaEventRecord(g_timing.ev[2 * slot_], st_);
    }
  }
  ~Timed() {
    if (slot_ >= 0) {
      cudaEventRecord(g_timing.ev[2 * slot_ + 1], st_);
      g_timing.sides[slot_] = kind_;
    }
  }
  Timed(const Timed&) = delete;
  Timed& operator=(const Timed&) = delete;

 private:
  cudaStream_t st_;
  int kind_;
  int slot_ = -1;
};
// Device status word of the current call's workspace (for kernels that report timeouts).
thread_local int* g_status_ptr = nullptr;

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

int g_num_sms = 0;
int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      g_num_sms = n;
    else
      return 152;
  }
  return g_num_sms;
}

struct Shape {
  int N = 0;
  int64_t I[kMaxOrder] = {};
  int64_t total = 0;
};

cpg_status check_shape(const int64_t* I, int N, int R, Shape& s) {
  if (I == nullptr || N < 2 || N > kMaxOrder || R < 1 || R > CPG_MAX_RANK) return CPG_ERR_ARG;
  s.N = N;
  int64_t t = 1;
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1) return CPG_ERR_ARG;
    if (t > INT64_MAX / I[n]) return CPG_ERR_SHAPE;
    t *= I[n];
    s.I[n] = I[n];
  }
  s.total = t;
  return CPG_OK;
}

int64_t prod(const Shape& s, int b, int e) {
  int64_t p = 1;
  for (int m = b; m < e; ++m) p *= s.I[m];
  return p;
}

// n* of Algorithm 2 step 1 (1-based count of leading modes), clamped to [1, N-1].
int split_point(const Shape& s) {
  int best = 0;
  for (int n = 1; n <= s.N; ++n)
    if (prod(s, 0, n) <= prod(s, n, s.N)) best = n;
  return std::min(std::max(best, 1), s.N - 1);
}

bool is_f64(int prec) { return prec == CPG_FP64; }
bool prec_valid(int prec) { return prec >= CPG_FP32 && prec <= CPG_BF16X6; }
// Precisions of the iterative sweeps (CP_ALS, NTF, batched CP_ALS): those
// whose gradient stays within 1e-5 of the exact one at every size.  BF16 (one
// limb, about 2^-9) and BF16x3 (two limbs, about 2^-17 per element) are
// gradient-only: each sweep's solve would carry their error into the factors.
bool sweep_prec_ok(int prec) { return prec != CPG_BF16 && prec != CPG_BF16X3; }

// ---- leading-pass plan ----------------------------------------------------------
struct LeadPlan {
  bool tc = false;  // tensor-core kernel (split BF16 / TF32 products)
  int tc_prec = 0;  // kTcBf16x3, kTcBf16, kTcTf32x3 or kTcBf16x6 (lead_tc_dispatch.cuh)
  int RTP = 0;      // tensor-core rank tile
  int k = 0, sides = 0;
  int64_t J = 0, K = 0;
  int RTmax = 0, groups = 0;   // rank groups of at most RTmax columns
  int TJ = 0, TK = 0, nrt = 1;
  int nJb = 0, nKs = 0;
  int64_t Kc = 0;
  size_t rpart_elems = 0, lpart_elems = 0;
  // CUDA-core kernel: Khatri-Rao rows built once per pass (kr_rows_kernel).
  int RT = 0;                 // the instance's rank tile (stored ranks per group)
  bool wl_rank_major = false;
  size_t wr_elems = 0, wl_elems = 0;
};

SimtShape shape_for(int prec, int r, int sides) {
  return is_f64(prec) ? simt_shape_f64(r, sides) : simt_shape_f32(r, sides);
}

bool is_tc_prec(int prec) {
  return prec == CPG_BF16X3 || prec == CPG_BF16 || prec == CPG_TF32X3 || prec == CPG_BF16X6;
}
int tc_code(int prec) {
  return prec == CPG_BF16X3 ? kTcBf16x3 : prec == CPG_BF16 ? kTcBf16 : prec == CPG_TF32X3 ? kTcTf32x3 : kTcBf16x6;
}

// Grid over (J-blocks, K-splits): the K-split count that best fills `slots`
// resident CTAs, discounting CTAs that run only a few stages; at most
// max_per column chunks per CTA.
void choose_ksplit(LeadPlan& p, int slots, int64_t max_per = INT64_MAX) {
  const int64_t chunks = (p.K + p.TK - 1) / p.TK;
  double best = -1.0;
  int best_ks = 1;
  const int64_t max_ks = std::min<int64_t>(chunks, 65535);
  for (int64_t ks = 1; ks <= max_ks; ++ks) {
    const int64_t per = (chunks + ks - 1) / ks;
    const int64_t nks = (chunks + per - 1) / per;
    if (nks != ks || per > max_per) continue;
    const int64_t units = int64_t(p.nJb) * nks;
    if (units > 65535LL * 64) break;
    const int64_t waves = (units + slots - 1) / slots;
    const double eff = double(units) / double(waves * slots);
    const double stages = double(per * p.nrt);
    const double score = eff * stages / (stages + 1.5);
    if (score > best + 1e-9) {
      best = score;
      best_ks = int(nks);
    }
  }
  p.nKs = best_ks;
  p.Kc = ((chunks + p.nKs - 1) / p.nKs) * p.TK;
}

// Grid of a CUDA-core leading pass: J-blocks of nrt row tiles (the L side
// alone may take several; with the R side nrt = 1) times K-splits of `per`
// column chunks.  Minimises, in units of one stage's time on a full GPU,
//   waves * (stages per CTA + 1.5) + (partial-sum bytes written and read back)
// over the distinct (nrt, per) pairs; `slots` = resident CTAs on the GPU.
void choose_grid(LeadPlan& p, int R, int esize, int slots) {
  const int64_t tiles = (p.J + p.TJ - 1) / p.TJ;
  const int64_t chunks = (p.K + p.TK - 1) / p.TK;
  const double stage_bytes = double(p.TJ) * p.TK * esize;
  double best = 1e300;
  int64_t best_nrt = 1, best_per = chunks;
  auto consider = [&](int64_t nrt, int64_t per) {
    const int64_t nJb = (tiles + nrt - 1) / nrt, nKs = (chunks + per - 1) / per;
    const int64_t units = nJb * nKs;
    if (nJb > 65535 || nKs > 65535) return;
    const double waves = double((units + slots - 1) / slots);
    double partial = 0.0;
    if (p.sides & 1) partial += 2.0 * double(nKs) * R * double(p.J) * esize;
    if (p.sides & 2) partial += 2.0 * double(nJb) * R * double(p.K) * esize;
    const double cost = waves * (double(per * nrt) + 1.5) + partial / (double(slots) * stage_bytes);
    if (cost < best - 1e-9) {
      best = cost;
      best_nrt = nrt;
      best_per = per;
    }
  };
  // Distinct values of ceil(n / d) for d = 1..n (about 2 sqrt(n) of them).
  auto distinct_ceils = [](int64_t n) {
    std::vector<int64_t> v;
    for (int64_t d = 1; d <= n;) {
      const int64_t q = (n + d - 1) / d;
      v.push_back(q);
      d = (q > 1) ? (n + q - 2) / (q - 1) : n + 1;  // next d with a smaller quotient
    }
    return v;
  };
  const std::vector<int64_t> nrts = (p.sides == 2) ? distinct_ceils(tiles) : std::vector<int64_t>{1};
  const std::vector<int64_t> pers = distinct_ceils(chunks);
  for (int64_t nrt : nrts)
    for (int64_t per : pers) consider(nrt, per);
  p.nrt = int(best_nrt);
  p.nJb = int((tiles + best_nrt - 1) / best_nrt);
  p.nKs = int((chunks + best_per - 1) / best_per);
  p.Kc = best_per * p.TK;
}

// The split-TF32 kernel accumulates a CTA's whole contraction range in tensor
// memory, where each MMA's sum is rounded toward zero: its error grows about
// linearly with the range (3.6e-6 relative at 704 columns, 3e-5 at 6579 on
// the 100^4 workload).  Ranges are capped at this many contraction entries;
// the partial sums of the ranges are added in FP32 round-to-nearest.
constexpr int64_t kTf32MaxRun = 512;

LeadPlan plan_lead_tc(const Shape& s, int R, int k, int sides, int prec) {
  LeadPlan p;
  p.tc = true;
  p.tc_prec = tc_code(prec);
  p.k = k;
  p.sides = sides;
  p.J = prod(s, 0, k);
  p.K = prod(s, k, s.N);
  p.RTmax = 64;
  p.groups = (R + p.RTmax - 1) / p.RTmax;
  p.RTP = tc_rank_tile(std::min(R, p.RTmax));
  p.TJ = tc_tile_rows(p.tc_prec, sides);
  p.TK = tc_tile_cols(p.tc_prec, sides);
  const int64_t tiles = (p.J + p.TJ - 1) / p.TJ;
  if (sides == 2) {
    // Step 7 alone: row tiles outer, one tensor-memory running sum per column
    // chunk (at most tc_max_acc chunks per CTA), W_L built once per row tile.
    // Minimise waves * (stages + W_L builds + fixed cost) + partial-sum
    // traffic, as choose_grid does for the CUDA-core kernel (1 CTA per SM).
    const int64_t max_per = std::max(1, tc_max_acc(p.RTP, 2, p.tc_prec));
    const int64_t max_nrt = p.tc_prec == kTcTf32x3 ? std::max<int64_t>(1, kTf32MaxRun / p.TJ) : tiles;
    const int64_t chunks = (p.K + p.TK - 1) / p.TK;
    const int slots = num_sms();
    const double wbuild = 0.25 * p.RTP / 16.0;  // one W_L build, in super-stages
    double best = 1e300;
    int64_t best_nrt = 1, best_per = 1;
    std::vector<int64_t> nrts;
    for (int64_t d = 1; d <= tiles;) {
      const int64_t q = (tiles + d - 1) / d;
      nrts.push_back(q);
      d = (q > 1) ? (tiles + q - 2) / (q - 1) : tiles + 1;
    }
    for (int64_t nrt : nrts)
      for (int64_t per = 1; per <= std::min(max_per, chunks) && nrt <= max_nrt; ++per) {
        const int64_t nJb = (tiles + nrt - 1) / nrt, nCb = (chunks + per - 1) / per;
        if (nJb > 65535 || nCb > 65535) continue;
        const double waves = double((nJb * nCb + slots - 1) / slots);
        const double partial = 2.0 * double(nJb) * R * double(p.K) * 4.0;
        const double stage_bytes = double(p.TJ) * p.TK * 4.0;
        const double cost = waves * (double(per * nrt) + double(nrt) * wbuild + 2.0) + partial / (double(slots) * stage_bytes);
        if (cost < best - 1e-9) {
          best = cost;
          best_nrt = nrt;
          best_per = per;
        }
      }
    p.nrt = int(best_nrt);
    p.nJb = int((tiles + best_nrt - 1) / best_nrt);
    p.nKs = int((chunks + best_per - 1) / best_per);
    p.Kc = best_per * p.TK;
  } else {
    const int cap = sides == 3 ? tc_fused_max_nrt(p.RTP, p.tc_prec) : std::min(tc_max_acc(p.RTP, 1, p.tc_prec), 8);
    p.nrt = int(std::max<int64_t>(1, std::min<int64_t>(tiles, cap)));
    p.nJb = int((p.J + int64_t(p.TJ) * p.nrt - 1) / (int64_t(p.TJ) * p.nrt));
    choose_ksplit(p, num_sms(), p.tc_prec == kTcTf32x3 ? std::max<int64_t>(1, kTf32MaxRun / p.TK) : INT64_MAX);
  }
  p.rpart_elems = (sides & 1) ? size_t(p.nKs) * R * p.J : 0;
  p.lpart_elems = (sides & 2) ? size_t(p.nJb) * R * p.K : 0;
  // Prebuilt B tiles of the split-BF16 passes (in the W row tables' place).
  size_t rb = 0, lb = 0;
  tc_wimg_bytes(p.RTP, sides, p.tc_prec, p.J, p.K, p.nrt, &rb, &lb);
  p.wr_elems = (rb + 3) / 4;
  p.wl_elems = (lb + 3) / 4;
  return p;
}

LeadPlan plan_lead(const Shape& s, int R, int k, int sides, int prec) {
  // Split-BF16 forms run on the tensor cores.
  if (is_tc_prec(prec)) return plan_lead_tc(s, R, k, sides, prec);
  LeadPlan p;
  p.k = k;
  p.sides = sides;
  p.J = prod(s, 0, k);
  p.K = prod(s, k, s.N);
  p.RTmax = is_f64(prec) ? kMaxRankTileF64 : kMaxRankTileF32;
  // FP32 step 4 copies Khatri-Rao rows built once per pass only up to rank 32
  // (above, a stage's rows outweigh half its tile and every CTA generates its
  // own: 0.33 TB/s at R = 64 on 60^5, against 2.7 TB/s at R = 32), and step 7
  // keeps two columns per lane only up to rank 32 (0.96 TB/s at R = 64,
  // 2.6 TB/s at R = 32).  Wider ranks run as balanced groups of at most 32,
  // one pass over Y each.
  if (!is_f64(prec) && (sides == 1 || sides == 2) && R > 32) {
    const int ng = (R + 31) / 32;
    p.RTmax = (R + ng - 1) / ng;
  }
  p.groups = (R + p.RTmax - 1) / p.RTmax;
  // All rank groups share one tile geometry: the widest group's.
  const SimtShape sh = shape_for(prec, std::min(R, p.RTmax), sides);
  p.TJ = sh.TJ;
  p.TK = sh.TK;
  const int bps = is_f64(prec) ? lead_blocks_per_sm_f64(sh.RT, sides) : lead_blocks_per_sm_f32(sh.RT, sides);
  choose_grid(p, R, is_f64(prec) ? 8 : 4, num_sms() * std::max(bps, 1));
  p.rpart_elems = (sides & 1) ? size_t(p.nKs) * R * p.J : 0;
  p.lpart_elems = (sides & 2) ? size_t(p.nJb) * R * p.K : 0;
  // Built rows: every column chunk (W_R) / row tile of every J-block (W_L) a CTA reads.
  p.RT = sh.RT;
  p.wl_rank_major = sh.wl_rank_major;
  p.wr_elems = (sh.wpre && (sides & 1)) ? size_t(p.groups) * p.RT * size_t((p.K + p.TK - 1) / p.TK * p.TK) : 0;
  p.wl_elems = (sh.wpre && (sides & 2)) ? size_t(p.groups) * p.RT * size_t(p.nJb) * p.nrt * p.TJ : 0;
  return p;
}

// ---- workspace ------------------------------------------------------------------
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename U>
  U* take(size_t n) {
    U* p = base ? reinterpret_cast<U*>(base + off) : nullptr;
    off = align_up(off + n * sizeof(U));
    return p;
  }
};

// First kAlign bytes of every workspace: the device status word, ||Y||^2,
// and the CTA ticket of the fused ALS mode kernels.
struct Header {
  int* status;
  double* normY2;
  unsigned int* ticket;
};

Header take_header(Carver& c) {
  Header h;
  char* p = c.take<char>(kAlign);
  h.status = reinterpret_cast<int*>(p);
  h.normY2 = p ? reinterpret_cast<double*>(p + 8) : nullptr;
  h.ticket = p ? reinterpret_cast<unsigned int*>(p + 16) : nullptr;
  return h;
}

template <typename T>
struct ChainBufs {
  T* Pa = nullptr;
  T* Pb = nullptr;
  T* Qa = nullptr;
  T* Qb = nullptr;
  T* kr = nullptr;
};

// Kronecker tables of the leading pass's Khatri-Rao rows (modes (0, k) for
// W_L and (k, N) for W_R; only needed when a run has three or more modes).
// Built Khatri-Rao rows of the CUDA-core passes (sized by the plans a:, b:).
template <typename T>
struct LeadTabs {
  T* qL = nullptr;
  T* qR = nullptr;
  T* wR = nullptr;
  T* wL = nullptr;
};

template <typename T>
LeadTabs<T> take_tabs(Carver& c, const Shape& s, int R, int k, const LeadPlan& a, const LeadPlan& b) {
  LeadTabs<T> t;
  t.qL = c.take<T>(size_t(R) * (k >= 3 ? prod(s, 1, k) : 1));
  t.qR = c.take<T>(size_t(R) * (s.N - k >= 3 ? prod(s, k + 1, s.N) : 1));
  t.wR = c.take<T>(std::max<size_t>(std::max(a.wr_elems, b.wr_elems), 1));
  t.wL = c.take<T>(std::max<size_t>(std::max(a.wl_elems, b.wl_elems), 1));
  return t;
}

int64_t kr_len_max(const Shape& s, int k) {
  // Longest Kronecker vector the chains build: modes [0, n-1) for n <= k, or
  // modes (n, N) for n >= k.
  int64_t m = 1;
  for (int n = 1; n <= k; ++n) m = std::max(m, prod(s, 0, n - 1));
  for (int n = k; n < s.N; ++n) m = std::max(m, prod(s, n + 1, s.N));
  return m;
}

template <typename T>
ChainBufs<T> take_chain(Carver& c, const Shape& s, int R, int64_t J, int64_t K, int k) {
  ChainBufs<T> b;
  b.Pa = c.take<T>(size_t(R) * J);
  b.Pb = c.take<T>(size_t(R) * J);
  b.Qa = c.take<T>(size_t(R) * K);
  b.Qb = c.take<T>(size_t(R) * K);
  b.kr = c.take<T>(size_t(R) * kr_len_max(s, k));
  return b;
}

struct GradLayout {
  LeadPlan lead;
  size_t bytes = 0;
};

// Row pitch (elements) of a copy of Y_(1:k) whose columns start on 16-byte
// boundaries, and its size; 0 when Y's own pitch J already does.
int64_t pitched_ld(int64_t J, size_t esize) {
  const int64_t q = int64_t(16 / esize);
  return (J + q - 1) / q * q;
}
size_t pitched_elems(int64_t J, int64_t K, size_t esize) {
  return (J * int64_t(esize)) % 16 == 0 ? 0 : size_t(pitched_ld(J, esize)) * size_t(K);
}

template <typename T>
struct GradWs {
  Header h;
  T* Rpart;
  T* Lpart;
  ChainBufs<T> ch;
  LeadTabs<T> tabs;
  T* Yp;  // Y_(1:k) with a 16-byte column pitch (yp_elems > 0), last in the layout
};

template <typename T>
GradWs<T> carve_grad(void* base, const Shape& s, int R, const LeadPlan& lp, size_t* bytes, size_t yp_elems = 0) {
  Carver c(base);
  GradWs<T> w;
  w.h = take_header(c);
  w.Rpart = c.take<T>(std::max<size_t>(lp.rpart_elems, 1));
  w.Lpart = c.take<T>(std::max<size_t>(lp.lpart_elems, 1));
  w.ch = take_chain<T>(c, s, R, lp.J, lp.K, lp.k);
  w.tabs = take_tabs<T>(c, s, R, lp.k, lp, lp);
  w.Yp = yp_elems ? c.take<T>(yp_elems) : nullptr;
  if (bytes) *bytes = c.off;
  return w;
}

// Fused pass unless its J-block partials would cost more than a fifth of Y's
// bytes; then the two sides run as separate passes (the L pass with tall blocks).
// The CUDA-core kernels fuse only at rank <= 4: with both sides a lane carries
// 2R products per element and too many accumulators for two CTAs per SM (at
// 100^4, R = 10 the fused pass ran at 2.0 TB/s against 5.1 and 4.2 TB/s for
// the single sides).
bool use_fused(const Shape& s, int R, int k, int prec) {
  if (is_tc_prec(prec) && !tc_fused_ok(tc_rank_tile(std::min(R, 64)), tc_code(prec))) return false;
  if (!is_tc_prec(prec) && R > 4) return false;
  const LeadPlan f = plan_lead(s, R, k, 3, prec);
  return double(f.lpart_elems + f.rpart_elems) <= 0.2 * double(s.total);
}

template <typename T>
struct ModeWs {
  Header h;
  T* part;
  T* kr;
  LeadTabs<T> tabs;
};

struct ModeRoute {
  bool right;
  LeadPlan lead;
};

ModeRoute mode_route(const Shape& s, int R, int n, int prec) {
  ModeRoute m;
  // Section 3.2: right-to-left (eq. 3.7) when J_n <= K_{n-1} (1-based), else left-to-right.
  m.right = prod(s, 0, n + 1) <= prod(s, n, s.N);
  m.lead = m.right ? plan_lead(s, R, n + 1, 1, prec) : plan_lead(s, R, n, 2, prec);
  return m;
}

template <typename T>
ModeWs<T> carve_mode(void* base, const Shape& s, int R, int n, const ModeRoute& rt, size_t* bytes) {
  Carver c(base);
  ModeWs<T> w;
  w.h = take_header(c);
  w.part = c.take<T>(std::max<size_t>(rt.right ? rt.lead.rpart_elems : rt.lead.lpart_elems, 1));
  const int64_t len = rt.right ? prod(s, 0, n) : prod(s, n + 1, s.N);
  w.kr = c.take<T>(size_t(R) * len);
  w.tabs = take_tabs<T>(c, s, R, rt.lead.k, rt.lead, rt.lead);
  if (bytes) *bytes = c.off;
  return w;
}

template <typename T>
struct AlsWs {
  Header h;
  T* Rpart;
  T* Lpart;
  double* normpart;
  ChainBufs<T> ch;
  double* grams;
  double* X;
  T* G;
  LeadTabs<T> tabs;
  double* V;   // [R][R] V of the current mode (double-float pairs for FP32 data)
  double* Vi;  // [R][R] V^{-1}
  T* Yp;       // Y_(1:k) with a 16-byte column pitch (yp_elems > 0), last in the layout
};

template <typename T>
AlsWs<T> carve_als(void* base, const Shape& s, int R, const LeadPlan& lr, const LeadPlan& ll, size_t* bytes,
                   size_t yp_elems = 0) {
  Carver c(base);
  AlsWs<T> w;
  w.h = take_header(c);
  w.Rpart = c.take<T>(std::max<size_t>(lr.rpart_elems, 1));
  w.Lpart = c.take<T>(std::max<size_t>(ll.lpart_elems, 1));
  w.normpart = c.take<double>(size_t(lr.nJb) * lr.nKs);
  w.ch = take_chain<T>(c, s, R, lr.J, lr.K, lr.k);
  int64_t imax = 1;
  for (int n = 0; n < s.N; ++n) imax = std::max(imax, s.I[n]);
  w.grams = c.take<double>(size_t(s.N) * R * R);
  w.X = c.take<double>(size_t(imax) * R);
  w.G = c.take<T>(size_t(imax) * R);
  w.tabs = take_tabs<T>(c, s, R, lr.k, lr, ll);
  w.V = c.take<double>(size_t(R) * R);
  w.Vi = c.take<double>(size_t(R) * R);
  w.Yp = yp_elems ? c.take<T>(yp_elems) : nullptr;
  if (bytes) *bytes = c.off;
  return w;
}

// Y_(1:k) into Yp with pitch pitched_ld(J): returns the tensor the leading
// passes read and its pitch.
template <typename T>
const T* pitch_copy(const T* Y, T* Yp, int64_t J, int64_t K, int64_t* ldy, cudaStream_t st) {
  if (Yp == nullptr) {
    *ldy = J;
    return Y;
  }
  *ldy = pitched_ld(J, sizeof(T));
  ++g_launches;
  Timed timer(st, kKindPitch);
  launch_pdl(pitch_copy_kernel<T>, dim3(unsigned(std::min<int64_t>(K, int64_t(16) * num_sms()))), dim3(256), 0, st, Yp,
             *ldy, Y, J, K);
  return Yp;
}

// Streams of a device's pool for batched calls.
constexpr int kPoolStreams = 16;

inline int blocks_for(int64_t n, int threads, int cap = 4 * 1024) {
  int64_t b = (n + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(b, cap)));
}

template <typename T>
FacArgs<T> fac_args(const Shape& s, const void* const* A) {
  FacArgs<T> f{};
  for (int m = 0; m < s.N; ++m) {
    f.I[m] = s.I[m];
    f.A[m] = static_cast<const T*>(A[m]);
  }
  return f;
}

// Kronecker vector over modes [mb, me) (eq. 3.3), [r][o] layout.  For a single
// mode it is the factor itself (column-major I x R has the same layout).
template <typename T>
const T* kr_vector(const Shape& s, const void* const* A, int R, int mb, int me, T* scratch, cudaStream_t st) {
  if (me - mb <= 0) return nullptr;
  if (me - mb == 1) return static_cast<const T*>(A[mb]);
  const int64_t len = prod(s, mb, me);
  ++g_launches;
  Timed timer(st, kKindKron);
  launch_pdl(kr_build_kernel<T>, dim3(blocks_for(len * R, 256)), dim3(256), 0, st, scratch, fac_args<T>(s, A), mb, me,
             len, R);
  return scratch;
}

// ---- launches -------------------------------------------------------------------
template <typename T>
cudaError_t launch_lead(const LeadArgs<T>& a, int RT, int sides, dim3 g, cudaStream_t st) {
  ++g_launches;
  Timed timer(st, sides);
  if constexpr (sizeof(T) == 8) return launch_lead_f64(a, RT, sides, g, st);
  else return launch_lead_f32(a, RT, sides, g, st);
}

// Khatri-Rao rows over modes [mb, me) as factor row x Kronecker-table entry.
template <typename T>
KrRows<T> make_rows(const Shape& s, const void* const* A, int R, int mb, int me, T* tab, cudaStream_t st) {
  KrRows<T> w;
  if (me <= mb) return w;
  w.A = static_cast<const T*>(A[mb]);
  w.d = FastDiv::make(uint32_t(s.I[mb]));
  w.Q = kr_vector<T>(s, A, R, mb + 1, me, tab, st);
  w.ldq = prod(s, mb + 1, me);
  return w;
}

template <typename T>
cudaError_t run_lead(const Shape& s, const T* Y, const void* const* A, int R, const LeadPlan& p, T* Rpart, T* Lpart,
                     double* normpart, int prec, const LeadTabs<T>& tabs, cudaStream_t st, int64_t ldy = 0) {
  if (ldy == 0) ldy = p.J;
  if constexpr (std::is_same_v<T, float>) {
    if (p.tc) {
      TcArgs a{};
      a.J = p.J;
      a.K = p.K;
      a.ldy = ldy;
      a.R = R;
      if (p.sides & 2) a.wl = make_rows<float>(s, A, R, 0, p.k, tabs.qL, st);
      if (p.sides & 1) a.wr = make_rows<float>(s, A, R, p.k, s.N, tabs.qR, st);
      a.Kc = p.Kc;
      a.nrt = p.nrt;
      a.Rpart = Rpart;
      a.Lpart = Lpart;
      a.status = g_status_ptr;
      a.wimg_r = reinterpret_cast<unsigned char*>(tabs.wR);
      a.wimg_l = reinterpret_cast<unsigned char*>(tabs.wL);
      for (int g = 0; g < p.groups; ++g) {
        a.r0 = g * p.RTmax;
        a.normpart = (g == 0) ? normpart : nullptr;
        cudaError_t e;
        if (p.wr_elems + p.wl_elems > 0) {
          g_launches += ((p.sides & 1) ? 1 : 0) + ((p.sides & 2) ? 1 : 0);
          Timed timer(st, kKindRows);
          e = launch_lead_tc_prep(a, p.RTP, p.sides, p.tc_prec, num_sms(), st);
          if (e != cudaSuccess) return e;
        }
        ++g_launches;
        {
          Timed timer(st, p.sides);
          e = launch_lead_tc(Y, a, p.RTP, p.sides, p.tc_prec, dim3(p.nJb, p.nKs), st);
        }
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    }
  }
  LeadArgs<T> a{};
  a.Y = Y;
  a.J = p.J;
  a.K = p.K;
  a.ldy = ldy;
  a.R = R;
  if (p.sides & 2) a.wl = make_rows<T>(s, A, R, 0, p.k, tabs.qL, st);
  if (p.sides & 1) a.wr = make_rows<T>(s, A, R, p.k, s.N, tabs.qR, st);
  a.Kc = p.Kc;
  a.nrt = p.nrt;
  a.Rpart = Rpart;
  a.Lpart = Lpart;
  a.status = g_status_ptr;
  // Every rank group runs the widest group's instance; ranks beyond R are masked.
  const int RT = p.RT;
  // Khatri-Rao rows built once per pass when the tiles come by TMA (the
  // kernel copies them with each tile); else every CTA generates its own.
  const bool wpre = matrix_map_ok(Y, int(sizeof(T)), p.J, p.K, ldy) && ((p.sides & 1) == 0 || p.wr_elems > 0) &&
                    ((p.sides & 2) == 0 || p.wl_elems > 0);
  const int64_t kpad = (p.K + p.TK - 1) / p.TK * p.TK, jpad = int64_t(p.nJb) * p.nrt * p.TJ;
  auto build = [&](T* dst, const KrRows<T>& kr, int64_t len, int64_t len_pad, int r0, int rank_major) {
    ++g_launches;
    Timed timer(st, kKindRows);
    const int64_t total = len_pad * RT;
    return launch_pdl(kr_rows_kernel<T>, dim3(blocks_for(total, 256, 2 * num_sms())), dim3(256), 0, st, dst, kr, len,
                      len_pad, RT, r0, R, p.TJ, rank_major);
  };
  for (int g = 0; g < p.groups; ++g) {
    a.r0 = g * p.RTmax;
    a.normpart = (g == 0) ? normpart : nullptr;
    a.wpre_r = nullptr;
    a.wpre_l = nullptr;
    if (wpre) {
      cudaError_t e = cudaSuccess;
      if (p.sides & 1) {
        T* d = tabs.wR + size_t(g) * RT * kpad;
        e = build(d, a.wr, p.K, kpad, a.r0, 0);
        a.wpre_r = d;
      }
      if (e == cudaSuccess && (p.sides & 2)) {
        T* d = tabs.wL + size_t(g) * RT * jpad;
        e = build(d, a.wl, p.J, jpad, a.r0, p.wl_rank_major ? 1 : 0);
        a.wpre_l = d;
      }
      if (e != cudaSuccess) return e;
    }
    cudaError_t e = launch_lead(a, RT, p.sides, dim3(p.nJb, p.nKs), st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The leading pass's partial sums, when there are enough of them, summed by
// a grid over the whole GPU before the chain: the first finishing contraction
// would otherwise add them up itself with a grid sized by its few outputs
// (15 x R at 15^7, where that took 150 us of a 470 us sweep).  Returns the
// tensor the chain reads and sets *nparts to 1, or leaves both unchanged.
constexpr int64_t kPresumMin = int64_t(1) << 20;  // elements read (all parts)

template <typename T>
const T* presum_parts(const T* X, int* nparts, int64_t n, T* out, cudaStream_t st) {
  if (*nparts <= 1 || int64_t(*nparts) * n < kPresumMin) return X;
  ++g_launches;
  Timed timer(st, kKindChain);
  launch_pdl(sum_parts_kernel<T>, dim3(blocks_for(n, 256, 8 * num_sms())), dim3(256), 0, st, out, X, *nparts, n, n);
  *nparts = 1;
  return out;
}

// Lanes per output of a segmented dot product of reduction length `inner`.
inline int seg_lanes(int64_t inner) { return inner >= 96 ? 32 : inner >= 24 ? 8 : inner >= 4 ? 4 : 1; }

template <typename T>
void launch_seg(const SegDot<T>& p, cudaStream_t st) {
  ++g_launches;
  Timed timer(st, kKindChain);
  const int64_t nout = p.D * p.R;
  auto go = [&](auto kern, int lpo) {
    const int64_t threads = nout * lpo;
    const int blocks = int(std::max<int64_t>(1, (threads + 255) / 256));
    launch_pdl(kern, dim3(blocks), dim3(256), 0, st, p);
  };
  if (seg_use_tiled(p)) {
    launch_pdl(seg_dot_tiled_kernel<T>, dim3(int(seg_tiled_blocks(p))), dim3(kSegWarps * 32), 0, st, p);
    return;
  }
  switch (seg_lanes(p.inner)) {
    case 32: go(seg_dot_kernel<T, 32>, 32); break;
    case 8: go(seg_dot_kernel<T, 8>, 8); break;
    case 4: go(seg_dot_kernel<T, 4>, 4); break;
    default: go(seg_dot_kernel<T, 1>, 1); break;
  }
}

// Finishing contraction for mode i of X (RIGHT: flat = o + len_o*i, LEFT: flat = i + In*o):
// G[i + In r] = sum_o X[r][flat] kr[r][o].
template <typename T, bool RIGHT>
SegDot<T> grad_seg(const T* X, int nparts, int64_t pstride, int64_t len_o, int64_t In, int R, const T* kr, T* G,
                   T* Xred) {
  SegDot<T> p{};
  p.X = X;
  p.nparts = nparts;
  p.part_stride = pstride;
  p.S = len_o * In;
  p.D = In;
  p.astep = RIGHT ? len_o : 1;
  p.ustep = RIGHT ? 1 : In;
  p.inner = len_o;
  p.w = kr;
  p.wlen = len_o;
  p.out = G;
  p.Xred = (nparts > 1) ? Xred : nullptr;
  p.R = R;
  return p;
}

template <typename T, bool RIGHT>
void launch_grad(const T* X, int nparts, int64_t pstride, int64_t len_o, int64_t In, int R, const T* kr, T* G, T* Xred,
                 cudaStream_t st) {
  launch_seg(grad_seg<T, RIGHT>(X, nparts, pstride, len_o, In, R, kr, G, Xred), st);
}

// Recursion over mode i of X: Xout[r][o] = sum_i X[r][flat] A[i + In r].
template <typename T, bool RIGHT>
SegDot<T> contract_seg(const T* X, int64_t len_o, int64_t In, int R, const T* An, T* Xout) {
  SegDot<T> p{};
  p.X = X;
  p.nparts = 1;
  p.part_stride = 0;
  p.S = len_o * In;
  p.D = len_o;
  p.astep = RIGHT ? 1 : In;
  p.ustep = RIGHT ? len_o : 1;
  p.inner = In;
  p.w = An;
  p.wlen = In;
  p.out = Xout;
  p.Xred = nullptr;
  p.R = R;
  return p;
}

template <typename T, bool RIGHT>
void launch_contract(const T* X, int64_t len_o, int64_t In, int R, const T* An, T* Xout, cudaStream_t st) {
  launch_seg(contract_seg<T, RIGHT>(X, len_o, In, R, An, Xout), st);
}

// One fused ALS mode (FP32 data): the segmented dot that produces G, then
// the update of mode u.n by the CTA that finishes last.
void launch_mode_update(const SegDot<float>& sd, const AlsDfArgs& u, unsigned int* ticket, cudaStream_t st) {
  ++g_launches;
  Timed timer(st, kKindMode);
  AlsModeArgs p{sd, u, ticket};
  const bool tiled = seg_use_tiled(sd);
  static_assert(kModeThreads == kSegWarps * 32, "the tiled segmented dot runs on mode-kernel blocks");
  const int lpo = tiled ? 0 : seg_lanes(sd.inner);
  const int64_t threads = sd.D * sd.R * std::max(lpo, 1);
  const int64_t seg_blocks = tiled ? seg_tiled_blocks(sd) : std::max<int64_t>(1, (threads + kModeThreads - 1) / kModeThreads);
  const int blocks = int(seg_blocks + 1);  // + the inverse CTA
  const size_t smem = als_df_smem_bytes(u.In, u.R);
  auto go = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    launch_pdl(kern, dim3(blocks), dim3(kModeThreads), smem, st, p);
  };
  switch (lpo) {
    case 0: go(als_mode_df_kernel<0>); break;
    case 32: go(als_mode_df_kernel<32>); break;
    case 8: go(als_mode_df_kernel<8>); break;
    case 4: go(als_mode_df_kernel<4>); break;
    default: go(als_mode_df_kernel<1>); break;
  }
}

cpg_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CPG_OK : CPG_ERR_CUDA; }

cpg_status common_checks(const cpg_opts* opts, Shape& s, const int64_t* I, int N, int R) {
  if (opts == nullptr) return CPG_ERR_ARG;
  cpg_status st = check_shape(I, N, R, s);
  if (st != CPG_OK) return st;
  if (!prec_valid(opts->precision)) return CPG_ERR_ARG;
  if (opts->split != 0 && (opts->split < 1 || opts->split > N - 1)) return CPG_ERR_ARG;
  return CPG_OK;
}

// The leading kernels index rows and columns with 32-bit arithmetic.
bool lead_fits(const LeadPlan& p) { return p.J < (int64_t(1) << 31) && p.K < (int64_t(1) << 31); }

int choose_split(const Shape& s, const cpg_opts* opts) {
  return (opts && opts->split != 0) ? opts->split : split_point(s);
}

// ---- plan of the all-mode gradient: split k, one fused pass or two ----------------
// One workspace layout for the two passes of a gradient: the R pass's plan
// with the larger of the two passes' L-side buffers.
LeadPlan grad_sizing(const LeadPlan& pr, const LeadPlan& pl) {
  LeadPlan z = pr;
  z.lpart_elems = std::max(pr.lpart_elems, pl.lpart_elems);
  z.wl_elems = std::max(pr.wl_elems, pl.wl_elems);
  return z;
}

struct GradChoice {
  int k = 1;
  bool fused = false;
};

// Workspace bytes of the all-mode gradient under plan c.
size_t grad_bytes(const Shape& s, int R, int prec, const GradChoice& c, bool with_copy = true) {
  LeadPlan pr = plan_lead(s, R, c.k, c.fused ? 3 : 1, prec);
  if (!c.fused) pr = grad_sizing(pr, plan_lead(s, R, c.k, 2, prec));
  const size_t ypn = (c.fused || !with_copy) ? 0 : pitched_elems(pr.J, pr.K, is_f64(prec) ? 8 : 4);
  size_t bytes = 0;
  if (is_f64(prec)) carve_grad<double>(nullptr, s, R, pr, &bytes, ypn);
  else carve_grad<float>(nullptr, s, R, pr, &bytes, ypn);
  return bytes;
}

// The planner's choice: n* (or the requested split) and the fused pass where
// use_fused allows it.
GradChoice default_choice(const Shape& s, int R, const cpg_opts* o) {
  GradChoice c;
  c.k = choose_split(s, o);
  c.fused = use_fused(s, R, c.k, o ? o->precision : CPG_FP32);
  return c;
}

// Plans the autotuner times: every split (or the requested one) x two passes,
// and the fused pass where the precision has one and its partial sums stay
// below the tensor's own size.
std::vector<GradChoice> grad_candidates(const Shape& s, int R, const cpg_opts* o) {
  std::vector<GradChoice> v;
  const int prec = o->precision;
  const int k0 = o->split != 0 ? o->split : 1, k1 = o->split != 0 ? o->split : s.N - 1;
  for (int k = k0; k <= k1; ++k) {
    GradChoice c;
    c.k = k;
    c.fused = false;
    v.push_back(c);
    if (!is_tc_prec(prec) || tc_fused_ok(tc_rank_tile(std::min(R, 64)), tc_code(prec))) {
      const LeadPlan f = plan_lead(s, R, k, 3, prec);
      if (double(f.lpart_elems + f.rpart_elems) <= double(s.total)) {
        c.fused = true;
        v.push_back(c);
      }
    }
  }
  return v;
}

// Measured plans (cpg_autotune_gradient), per device, precision, requested
// split, rank and shape.
std::map<std::vector<int64_t>, GradChoice> g_tuned;
std::mutex g_tuned_mu;

std::vector<int64_t> tune_key(const Shape& s, int R, const cpg_opts* o) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<int64_t> key = {dev, o ? o->precision : 0, o ? o->split : 0, R, s.N};
  for (int n = 0; n < s.N; ++n) key.push_back(s.I[n]);
  return key;
}

bool tuned_choice(const Shape& s, int R, const cpg_opts* o, GradChoice* c) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  auto it = g_tuned.find(tune_key(s, R, o));
  if (it == g_tuned.end()) return false;
  *c = it->second;
  return true;
}

// The plan cp_gradient_all runs: the measured one when there is one and the
// workspace holds it, else the planner's.
GradChoice grad_choice(const Shape& s, int R, const cpg_opts* o) {
  GradChoice c;
  // The measured plan whenever the workspace holds it, with or without room
  // for the pitched copy of Y (the call takes the copy only when it fits).
  if (tuned_choice(s, R, o, &c) && o->workspace_bytes >= grad_bytes(s, R, o->precision, c, false)) return c;
  return default_choice(s, R, o);
}

// ---- split of the CP_ALS sweep --------------------------------------------------------
// Workspace bytes of a CP_ALS (or NTF) sweep at split k.
size_t als_bytes(const Shape& s, int R, int prec, int k, bool with_copy) {
  const LeadPlan lr = plan_lead(s, R, k, 1, prec), ll = plan_lead(s, R, k, 2, prec);
  const size_t ypn = with_copy ? pitched_elems(lr.J, lr.K, is_f64(prec) ? 8 : 4) : 0;
  size_t bytes = 0;
  if (is_f64(prec)) carve_als<double>(nullptr, s, R, lr, ll, &bytes, ypn);
  else carve_als<float>(nullptr, s, R, lr, ll, &bytes, ypn);
  return bytes;
}

// Modelled cost of one sweep at split k (1-based count of leading modes), in
// elements moved: the two passes over Y (Algorithm 2 steps 4 and 7, the same
// for every k), the Khatri-Rao operands of the passes, and the recursions of
// steps 11 and 15 with their finishing contractions (steps 19 and 20), which
// read R^(m) (J_m x R, m <= k) and L^(m) (R x K_(m-1), m > k) and whose
// multiplication counts Table 4.1 sums the same way.  Partial results are
// written once and read once.
double als_model_cost(const Shape& s, int R, int k) {
  std::vector<double> J(s.N + 1, 1.0), K(s.N + 1, 1.0);  // J[m] = I_0..I_(m-1), K[m] = I_m..I_(N-1)
  for (int m = 1; m <= s.N; ++m) J[m] = J[m - 1] * double(s.I[m - 1]);
  for (int m = s.N - 1; m >= 0; --m) K[m] = K[m + 1] * double(s.I[m]);
  double side = J[k] + K[k];  // Khatri-Rao operands of the two passes
  for (int m = 1; m <= k; ++m) side += 2.0 * J[m];
  for (int m = k; m < s.N; ++m) side += 2.0 * K[m];
  return 2.0 * double(s.total) + double(R) * side;
}

// Splits the ALS autotuner times: opts->split alone when set, else n*
// (Algorithm 2 step 1) and every k whose modelled cost is within 1.25x of
// the cheapest, cheapest first.
std::vector<int> als_candidates(const Shape& s, int R, const cpg_opts* o) {
  if (o && o->split != 0) return {o->split};
  std::vector<std::pair<double, int>> c;
  double best = 0.0;
  for (int k = 1; k <= s.N - 1; ++k) {
    const double m = als_model_cost(s, R, k);
    c.push_back({m, k});
    if (k == 1 || m < best) best = m;
  }
  std::stable_sort(c.begin(), c.end());
  std::vector<int> v;
  for (const auto& e : c)
    if (e.first <= 1.25 * best || e.second == split_point(s)) v.push_back(e.second);
  return v;
}

// Measured splits (cpg_autotune_als), keyed like the gradient's plans.
std::map<std::vector<int64_t>, int> g_als_tuned;

bool tuned_als_split(const Shape& s, int R, const cpg_opts* o, int* k) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  auto it = g_als_tuned.find(tune_key(s, R, o));
  if (it == g_als_tuned.end()) return false;
  *k = it->second;
  return true;
}

// The split a sweep runs: the requested one, else the measured one when the
// workspace holds it, else n*.
int als_split(const Shape& s, int R, const cpg_opts* o) {
  if (o->split != 0) return o->split;
  int k = 0;
  if (tuned_als_split(s, R, o, &k) && o->workspace_bytes >= als_bytes(s, R, o->precision, k, false)) return k;
  return split_point(s);
}

// ---- all-mode gradient (Algorithm 2) ------------------------------------------------
template <typename T>
cpg_status gradient_all_impl(const Shape& s, const T* Y, const void* const* A, int R, void* const* G,
                             const cpg_opts* o, const GradChoice& plan) {
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  const int k = plan.k;
  const bool fused = plan.fused;
  LeadPlan pr = plan_lead(s, R, k, fused ? 3 : 1, o->precision);
  LeadPlan pl = fused ? pr : plan_lead(s, R, k, 2, o->precision);
  // Workspace: one layout sized for the larger of the two plans.
  const LeadPlan sizing = grad_sizing(pr, pl);
  // Two passes over a tensor whose column pitch is not a multiple of 16
  // bytes: a pitched copy (when the workspace holds it) lets both take TMA
  // tiles, for one extra read and write of Y.
  const size_t ypn = fused ? 0 : pitched_elems(pr.J, pr.K, sizeof(T));
  size_t need = 0, need_copy = 0;
  carve_grad<T>(nullptr, s, R, sizing, &need_copy, ypn);
  const bool copy_y = ypn > 0 && o->workspace != nullptr && o->workspace_bytes >= need_copy;
  GradWs<T> w = carve_grad<T>(o->workspace, s, R, sizing, &need, copy_y ? ypn : 0);
  if (!lead_fits(pr) || !lead_fits(pl)) return CPG_ERR_UNSUPPORTED;
  if (o->workspace == nullptr || o->workspace_bytes < need) return CPG_ERR_WORKSPACE;
  g_status_ptr = w.h.status;

  // Steps 4 and 7: R^(k) and L^(k+1) from one read of Y (or two passes).
  int64_t ldy = 0;
  const T* Yl = pitch_copy<T>(Y, w.Yp, pr.J, pr.K, &ldy, st);
  cudaError_t e = run_lead<T>(s, Yl, A, R, pr, w.Rpart, w.Lpart, nullptr, o->precision, w.tabs, st, ldy);
  if (e == cudaSuccess && !fused)
    e = run_lead<T>(s, Yl, A, R, pl, nullptr, w.Lpart, nullptr, o->precision, w.tabs, st, ldy);
  if (e != cudaSuccess) return CPG_ERR_CUDA;

  // Right side: modes k-1, ..., 0 (steps 5, 11, 12; finishing contraction line 19).
  {
    int nparts = pr.nKs;
    const int64_t pstride = int64_t(R) * pr.J;
    T* bufs[2] = {w.ch.Pa, w.ch.Pb};
    int cur = 0;
    const T* X = presum_parts<T>(w.Rpart, &nparts, pstride, bufs[cur], st);
    for (int n = k; n >= 1; --n) {
      const int m = n - 1;
      const int64_t len_o = prod(s, 0, m), In = s.I[m];
      const T* kr = kr_vector<T>(s, A, R, 0, m, w.ch.kr, st);
      T* Xred = (nparts > 1 && m > 0) ? bufs[cur] : nullptr;
      launch_grad<T, true>(X, nparts, pstride, len_o, In, R, kr, static_cast<T*>(G[m]), Xred, st);
      if (m > 0) {
        const T* src = Xred ? Xred : X;
        T* dst = bufs[cur ^ 1];
        launch_contract<T, true>(src, len_o, In, R, static_cast<const T*>(A[m]), dst, st);
        X = dst;
        nparts = 1;
        cur ^= 1;
      }
    }
  }
  // Left side: modes k, ..., N-1 (steps 8, 15, 16; finishing contraction line 20).
  {
    int nparts = pl.nJb;
    const int64_t pstride = int64_t(R) * pl.K;
    T* bufs[2] = {w.ch.Qa, w.ch.Qb};
    int cur = 0;
    const T* X = presum_parts<T>(w.Lpart, &nparts, pstride, bufs[cur], st);
    for (int n = k; n < s.N; ++n) {
      const int64_t len_o = prod(s, n + 1, s.N), In = s.I[n];
      const T* kr = kr_vector<T>(s, A, R, n + 1, s.N, w.ch.kr, st);
      T* Xred = (nparts > 1 && n < s.N - 1) ? bufs[cur] : nullptr;
      launch_grad<T, false>(X, nparts, pstride, len_o, In, R, kr, static_cast<T*>(G[n]), Xred, st);
      if (n < s.N - 1) {
        const T* src = Xred ? Xred : X;
        T* dst = bufs[cur ^ 1];
        launch_contract<T, false>(src, len_o, In, R, static_cast<const T*>(A[n]), dst, st);
        X = dst;
        nparts = 1;
        cur ^= 1;
      }
    }
  }
  return cuda_status(cudaGetLastError());
}

// ---- cost gradient of eq. 2.13, first-order step of eq. 2.15 -------------------------
// Workspace: the all-mode gradient's, then the FP64 Grams and Gamma^(n) in its
// last grams_bytes (at a 256-byte boundary).
inline size_t grams_bytes(int N, int R) { return 2 * align_up(size_t(N) * R * R * sizeof(double)); }

template <typename T>
cpg_status gradient_full_impl(const Shape& s, const T* Y, void* const* A, int R, void* const* G, const cpg_opts* o,
                              double eta, bool step) {
  const size_t gb = grams_bytes(s.N, R);
  if (o->workspace == nullptr || o->workspace_bytes < gb + kAlign) return CPG_ERR_WORKSPACE;
  cpg_opts og = *o;
  og.workspace_bytes = (o->workspace_bytes - gb) / kAlign * kAlign;
  double* grams = reinterpret_cast<double*>(static_cast<char*>(o->workspace) + og.workspace_bytes);
  double* gammas = reinterpret_cast<double*>(reinterpret_cast<char*>(grams) + gb / 2);
  // Y_(n) KR for every mode (Algorithm 2) at the current factors.
  const void* const* Ac = const_cast<const void* const*>(A);
  cpg_status st = gradient_all_impl<T>(s, Y, Ac, R, G, &og, grad_choice(s, R, &og));
  if (st != CPG_OK) return st;
  cudaStream_t str = static_cast<cudaStream_t>(o->stream);
  ++g_launches;
  {
    Timed timer(str, kKindGram);
    launch_pdl(gram_all_kernel<T>, dim3(blocks_for(int64_t(R) * R, 256), s.N), dim3(256), 0, str, fac_args<T>(s, Ac),
               R, grams);
  }
  ++g_launches;
  {
    Timed timer(str, kKindGram);
    launch_pdl(gamma_all_kernel, dim3(blocks_for(int64_t(R) * R, 256), s.N), dim3(256), 0, str,
               static_cast<const double*>(grams), s.N, R, gammas);
  }
  ModelTermArgs<T> a{};
  a.N = s.N;
  a.R = R;
  int64_t imax = 1;
  for (int n = 0; n < s.N; ++n) {
    a.I[n] = s.I[n];
    a.A[n] = static_cast<T*>(A[n]);
    a.G[n] = static_cast<T*>(G[n]);
    imax = std::max(imax, s.I[n]);
  }
  a.gammas = gammas;
  a.eta = eta;
  a.step = step ? 1 : 0;
  ++g_launches;
  {
    Timed timer(str, kKindModelTerm);
    launch_pdl(model_term_kernel<T>, dim3(blocks_for(imax, kRowsPerBlock, 1 << 30), s.N), dim3(256),
               size_t(kRowsPerBlock) * R * sizeof(double), str, a);
  }
  return cuda_status(cudaGetLastError());
}

// ---- single-mode gradient (Section 3.2) ----------------------------------------------
template <typename T>
cpg_status gradient_mode_impl(const Shape& s, const T* Y, const void* const* A, int R, int n, T* Gn,
                              const cpg_opts* o) {
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  const ModeRoute rt = mode_route(s, R, n, o->precision);
  size_t need = 0;
  ModeWs<T> w = carve_mode<T>(o->workspace, s, R, n, rt, &need);
  if (!lead_fits(rt.lead)) return CPG_ERR_UNSUPPORTED;
  if (o->workspace == nullptr || o->workspace_bytes < need) return CPG_ERR_WORKSPACE;
  g_status_ptr = w.h.status;
  const LeadPlan& p = rt.lead;
  if (rt.right) {
    // R^(n) = Y_(1:n) (KR over modes > n) (eq. 3.10), then eq. 3.12.
    if (run_lead<T>(s, Y, A, R, p, w.part, nullptr, nullptr, o->precision, w.tabs, st) != cudaSuccess) return CPG_ERR_CUDA;
    const T* kr = kr_vector<T>(s, A, R, 0, n, w.kr, st);
    launch_grad<T, true>(w.part, p.nKs, int64_t(R) * p.J, prod(s, 0, n), s.I[n], R, kr, Gn, nullptr, st);
  } else {
    // L^(n) = (KR over modes < n)^T Y_(1:n-1) (eq. 3.9), then eq. 3.16.
    if (run_lead<T>(s, Y, A, R, p, nullptr, w.part, nullptr, o->precision, w.tabs, st) != cudaSuccess) return CPG_ERR_CUDA;
    const T* kr = kr_vector<T>(s, A, R, n + 1, s.N, w.kr, st);
    launch_grad<T, false>(w.part, p.nJb, int64_t(R) * p.K, prod(s, n + 1, s.N), s.I[n], R, kr, Gn, nullptr, st);
  }
  return cuda_status(cudaGetLastError());
}

// ---- fast CP_ALS (Section 4) -------------------------------------------------------
constexpr int kAlsMaxRank = 64;

// mu = false: fast CP_ALS (eq. 2.14); mu = true: the same sweep with the
// multiplicative nonnegative update of eq. 2.18 in place of the solve (no
// normalisation, lambda unused).
template <typename T>
cpg_status als_impl(const Shape& s, const T* Y, void* const* A, double* lambda, int R, int iters, double* fit,
                    const cpg_opts* o, int* status_override = nullptr, bool mu = false) {
  cudaStream_t st = static_cast<cudaStream_t>(o->stream);
  if (R > kAlsMaxRank) return CPG_ERR_UNSUPPORTED;
  const int k = als_split(s, R, o);
  const LeadPlan lr = plan_lead(s, R, k, 1, o->precision);
  const LeadPlan ll = plan_lead(s, R, k, 2, o->precision);
  // A copy of Y with a 16-byte column pitch when Y's own pitch is not one and
  // the workspace holds it (cpg_workspace_size counts it): 2 * iters passes
  // then take TMA tiles, for one extra read and write of Y.
  const size_t ypn = pitched_elems(lr.J, lr.K, sizeof(T));
  size_t need = 0, need_copy = 0;
  carve_als<T>(nullptr, s, R, lr, ll, &need_copy, ypn);
  const bool copy_y = ypn > 0 && o->workspace != nullptr && o->workspace_bytes >= need_copy;
  AlsWs<T> w = carve_als<T>(o->workspace, s, R, lr, ll, &need, copy_y ? ypn : 0);
  if (!lead_fits(lr) || !lead_fits(ll)) return CPG_ERR_UNSUPPORTED;
  if (o->workspace == nullptr || o->workspace_bytes < need) return CPG_ERR_WORKSPACE;
  if (status_override) w.h.status = status_override;
  g_status_ptr = w.h.status;
  const void* const* Ac = const_cast<const void* const*>(A);

  constexpr bool kDf = std::is_same_v<T, float>;
  const bool fused = kDf && !mu;  // FP32 least squares: the fused mode kernels
  int64_t imax = 1;
  for (int m = 0; m < s.N; ++m) imax = std::max(imax, s.I[m]);
  constexpr size_t kSmemCap = 200 * 1024;
  const bool smem_path = (kDf ? als_df_smem_bytes(imax, R) : als_smem_bytes(imax, R)) <= kSmemCap;
  if (fused && !smem_path) return CPG_ERR_UNSUPPORTED;
  const size_t upd_smem = size_t(3) * R * R * sizeof(double);
  if constexpr (!kDf) {
    cudaFuncSetAttribute(als_update_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(upd_smem));
    if (smem_path)
      cudaFuncSetAttribute(als_update_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           int(als_smem_bytes(imax, R)));
  } else if (fused) {
    // The fused mode kernels' CTA ticket starts at zero.
    if (cudaMemsetAsync(w.h.ticket, 0, sizeof(unsigned int), st) != cudaSuccess) return CPG_ERR_CUDA;
  }

  ++g_launches;
  {
    // Double-float Grams for the fused FP32 path, FP64 otherwise.
    Timed timer(st, kKindGram);
    bool done = false;
    if constexpr (kDf) {
      if (fused) {
        launch_pdl(gram_all_df_kernel, dim3(blocks_for(int64_t(R) * R, 256), s.N), dim3(256), 0, st, fac_args<T>(s, Ac),
                   R, reinterpret_cast<df*>(w.grams));
        done = true;
      }
    }
    if (!done)
      launch_pdl(gram_all_kernel<T>, dim3(blocks_for(int64_t(R) * R, 256), s.N), dim3(256), 0, st, fac_args<T>(s, Ac),
                 R, w.grams);
  }

  // The update of mode n from G^(n) = Gn.  FP32 data: fused into the kernel
  // that produces G (sd, whose output is w.G); FP64 data: its own launch
  // after the G kernel.
  auto update = [&](int n, const SegDot<T>& sd, double* fit_out) {
    if constexpr (kDf) {
      if (!mu) {
        AlsDfArgs u{};
        u.N = s.N;
        u.n = n;
        u.R = R;
        u.In = s.I[n];
        u.grams = reinterpret_cast<df*>(w.grams);
        u.V = reinterpret_cast<df*>(w.V);
        u.Vi = reinterpret_cast<df*>(w.Vi);
        u.G = sd.out;
        u.An = static_cast<float*>(A[n]);
        u.lambda = lambda;
        u.status = w.h.status;
        u.fit_out = fit_out;
        u.normY2 = w.h.normY2;
        launch_mode_update(sd, u, w.h.ticket, st);
        return;
      }
    }
    const bool identity = sd.inner == 1 && sd.nparts == 1 && sd.X == sd.out;
    if (!identity) launch_seg(sd, st);
    ++g_launches;
    Timed timer(st, kKindUpdate);
    if (mu) {
      // eq. 2.18, then the Gram of the new factor (and the fit after the last mode).
      MuArgs<T> u{};
      u.N = s.N;
      u.n = n;
      u.R = R;
      u.In = s.I[n];
      u.grams = w.grams;
      u.G = sd.out;
      u.An = static_cast<T*>(A[n]);
      const size_t sm = size_t(R + kRowsPerBlock) * R * sizeof(double);
      launch_pdl(mu_update_kernel<T>, dim3(blocks_for(s.I[n], kRowsPerBlock, 1 << 30)), dim3(256), sm, st, u);
      FacArgs<T> f{};
      f.I[0] = s.I[n];
      f.A[0] = static_cast<const T*>(A[n]);
      ++g_launches;
      launch_pdl(gram_all_kernel<T>, dim3(blocks_for(int64_t(R) * R, 256), 1), dim3(256), 0, st, f, R,
                 w.grams + int64_t(n) * R * R);
      if (fit_out != nullptr) {
        ++g_launches;
        launch_pdl(ntf_fit_kernel<T>, dim3(1), dim3(256), 0, st, s.N, R, s.I[n], static_cast<const T*>(A[n]), sd.out,
                   static_cast<const double*>(w.grams), static_cast<const double*>(w.h.normY2), fit_out);
      }
      return;
    }
    if constexpr (!kDf) {
      AlsArgs<T> u{};
      u.N = s.N;
      u.n = n;
      u.R = R;
      u.In = s.I[n];
      u.grams = w.grams;
      u.G = sd.out;
      u.An = static_cast<T*>(A[n]);
      u.lambda = lambda;
      u.X = w.X;
      u.status = w.h.status;
      u.fit_out = fit_out;
      u.normY2 = w.h.normY2;
      if (smem_path)
        launch_pdl(als_update_smem_kernel<T>, dim3(1), dim3(512), als_smem_bytes(s.I[n], R), st, u);
      else
        launch_pdl(als_update_kernel<T>, dim3(1), dim3(256), upd_smem, st, u);
    }
  };
  // G^(n) of a mode whose finishing contraction is the identity (a single
  // remaining mode with no partial sums): X itself.  The fused FP32 path
  // copies it into w.G inside its mode kernel; the others read it in place.
  auto identity_seg = [&](const T* X, int64_t In) {
    SegDot<T> p{};
    p.X = X;
    p.nparts = 1;
    p.S = In;
    p.D = In;
    p.astep = 1;
    p.ustep = 1;
    p.inner = 1;
    p.out = fused ? w.G : const_cast<T*>(X);
    p.R = R;
    return p;
  };

  int64_t ldy = 0;
  const T* Yl = pitch_copy<T>(Y, w.Yp, lr.J, lr.K, &ldy, st);
  for (int it = 0; it < iters; ++it) {
    // Pass 1: R^(k) with the current trailing factors (step 4); modes k-1, ..., 0.
    double* np = (it == 0) ? w.normpart : nullptr;
    if (run_lead<T>(s, Yl, Ac, R, lr, w.Rpart, nullptr, np, o->precision, w.tabs, st, ldy) != cudaSuccess)
      return CPG_ERR_CUDA;
    if (it == 0) {
      ++g_launches;
      Timed timer(st, kKindNorm);
      launch_pdl(sum_norm_kernel, dim3(1), dim3(256), 0, st, w.normpart, int64_t(lr.nJb) * lr.nKs, w.h.normY2);
    }
    {
      int nparts = lr.nKs;
      const int64_t pstride = int64_t(R) * lr.J;
      T* bufs[2] = {w.ch.Pa, w.ch.Pb};
      int cur = 0;
      const T* X = presum_parts<T>(w.Rpart, &nparts, pstride, bufs[cur], st);
      bool g_done = false;  // this mode's update already ran (fused with the recursion)
      for (int n = k; n >= 1; --n) {
        const int m = n - 1;
        const int64_t len_o = prod(s, 0, m), In = s.I[m];
        T* Xred = nullptr;
        if (!g_done) {
          if (len_o == 1 && nparts == 1) {
            update(m, identity_seg(X, In), nullptr);
          } else {
            const T* kr = kr_vector<T>(s, Ac, R, 0, m, w.ch.kr, st);
            Xred = (nparts > 1 && m > 0) ? bufs[cur] : nullptr;
            update(m, grad_seg<T, true>(X, nparts, pstride, len_o, In, R, kr, w.G, Xred), nullptr);
          }
        }
        g_done = false;
        if (m > 0) {
          // Recursion with the updated a^(m) (eq. 3.20).  When the next mode is
          // mode 0, the contracted tensor is G^(0) itself: its update is fused.
          const T* src = Xred ? Xred : X;
          if (fused && m == 1) {
            update(0, contract_seg<T, true>(src, len_o, In, R, static_cast<const T*>(A[m]), w.G), nullptr);
            g_done = true;
          } else {
            T* dst = bufs[cur ^ 1];
            launch_contract<T, true>(src, len_o, In, R, static_cast<const T*>(A[m]), dst, st);
            X = dst;
            nparts = 1;
            cur ^= 1;
          }
        }
      }
    }
    // Pass 2: L^(k+1) with the updated leading factors (step 7); modes k, ..., N-1.
    if (run_lead<T>(s, Yl, Ac, R, ll, nullptr, w.Lpart, nullptr, o->precision, w.tabs, st, ldy) != cudaSuccess)
      return CPG_ERR_CUDA;
    {
      int nparts = ll.nJb;
      const int64_t pstride = int64_t(R) * ll.K;
      T* bufs[2] = {w.ch.Qa, w.ch.Qb};
      int cur = 0;
      const T* X = presum_parts<T>(w.Lpart, &nparts, pstride, bufs[cur], st);
      bool g_done = false;
      auto fit_of = [&](int n) { return (n == s.N - 1 && fit) ? fit + it : nullptr; };
      for (int n = k; n < s.N; ++n) {
        const int64_t len_o = prod(s, n + 1, s.N), In = s.I[n];
        T* Xred = nullptr;
        if (!g_done) {
          if (len_o == 1 && nparts == 1) {
            update(n, identity_seg(X, In), fit_of(n));
          } else {
            const T* kr = kr_vector<T>(s, Ac, R, n + 1, s.N, w.ch.kr, st);
            Xred = (nparts > 1 && n < s.N - 1) ? bufs[cur] : nullptr;
            update(n, grad_seg<T, false>(X, nparts, pstride, len_o, In, R, kr, w.G, Xred), fit_of(n));
          }
        }
        g_done = false;
        if (n < s.N - 1) {
          // Recursion with the updated a^(n) (eq. 3.22); fused with the update
          // of mode N-1 when that is the next mode.
          const T* src = Xred ? Xred : X;
          if (fused && n + 1 == s.N - 1) {
            update(n + 1, contract_seg<T, false>(src, len_o, In, R, static_cast<const T*>(A[n]), w.G), fit_of(n + 1));
            g_done = true;
          } else {
            T* dst = bufs[cur ^ 1];
            launch_contract<T, false>(src, len_o, In, R, static_cast<const T*>(A[n]), dst, st);
            X = dst;
            nparts = 1;
            cur ^= 1;
          }
        }
      }
    }
  }
  return cuda_status(cudaGetLastError());
}

// ---- failure detection ----------------------------------------------------------------
// One CTA waits on an mbarrier phase that nothing completes, with the bounded
// wait every kernel of this library uses; on expiry it records
// CPG_ERR_TIMEOUT in the status word and returns.
__global__ void timeout_selftest_kernel(int* status, uint32_t polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    tc::mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0u, polls)) atomicCAS(status, 0, int(CPG_ERR_TIMEOUT));
}

// ---- batched CP_ALS ------------------------------------------------------------------
struct StreamPool {
  cudaStream_t s[kPoolStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kPoolStreams] = {};
};

StreamPool* stream_pool() {
  static StreamPool table[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  StreamPool& p = table[dev];
  if (p.fork == nullptr) {
    for (int i = 0; i < kPoolStreams; ++i) {
      if (cudaStreamCreateWithFlags(&p.s[i], cudaStreamNonBlocking) != cudaSuccess) return nullptr;
      if (cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming) != cudaSuccess) return nullptr;
    }
    if (cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  }
  return &p;
}

// Per-member options with the member's workspace slice; 0 bytes on invalid members.
size_t member_ws_bytes(const cpg_tensor_desc& d, const cpg_opts* opts) {
  return cpg_workspace_size(d.I, d.N, d.R, opts, CPG_CALL_ALS);
}

bool ptrs_ok(const void* const* P, int N) {
  if (P == nullptr) return false;
  for (int n = 0; n < N; ++n)
    if (P[n] == nullptr) return false;
  return true;
}

// The ALS autotuner keeps the caller's factors and lambda after the largest
// candidate's workspace.
size_t als_tune_save_offset(size_t als_need) { return align_up(als_need); }
size_t als_tune_save_bytes(const Shape& s, int R, int prec) {
  size_t e = 0;
  for (int n = 0; n < s.N; ++n) e += size_t(s.I[n]) * size_t(R);
  return align_up(e * (is_f64(prec) ? 8 : 4)) + size_t(R) * sizeof(double);
}

// Workspace bytes of `call`; with_copy: including the optional pitched copy of Y.
size_t workspace_size_impl(const int64_t* I, int N, int R, const cpg_opts* opts, int call, bool with_copy) {
  Shape s;
  if (check_shape(I, N, R, s) != CPG_OK) return 0;
  const int prec = opts ? opts->precision : CPG_FP32;
  if (!prec_valid(prec)) return 0;
  if (opts && opts->split != 0 && (opts->split < 1 || opts->split > N - 1)) return 0;
  const int k = choose_split(s, opts);
  size_t bytes = 0;
  cpg_opts od{};
  if (opts) od = *opts;
  od.precision = prec;
  if (call == CPG_CALL_GRADIENT_ALL) {
    bytes = grad_bytes(s, R, prec, default_choice(s, R, &od), with_copy);
    GradChoice t;
    if (tuned_choice(s, R, &od, &t)) bytes = std::max(bytes, grad_bytes(s, R, prec, t, with_copy));
  } else if (call == CPG_CALL_GRADIENT_FULL) {
    bytes = grad_bytes(s, R, prec, default_choice(s, R, &od), with_copy);
    GradChoice t;
    if (tuned_choice(s, R, &od, &t)) bytes = std::max(bytes, grad_bytes(s, R, prec, t, with_copy));
    bytes = align_up(bytes) + grams_bytes(N, R) + kAlign;
  } else if (call == CPG_CALL_GRADIENT_TUNE) {
    for (const GradChoice& c : grad_candidates(s, R, &od)) bytes = std::max(bytes, grad_bytes(s, R, prec, c, with_copy));
  } else if (call == CPG_CALL_GRADIENT_MODE) {
    for (int n = 0; n < N; ++n) {
      size_t b = 0;
      const ModeRoute rt = mode_route(s, R, n, prec);
      if (is_f64(prec)) carve_mode<double>(nullptr, s, R, n, rt, &b);
      else carve_mode<float>(nullptr, s, R, n, rt, &b);
      bytes = std::max(bytes, b);
    }
  } else if (call == CPG_CALL_ALS || call == CPG_CALL_NTF) {
    bytes = als_bytes(s, R, prec, k, with_copy);
    int t = 0;
    if ((!opts || opts->split == 0) && tuned_als_split(s, R, &od, &t))
      bytes = std::max(bytes, als_bytes(s, R, prec, t, with_copy));
  } else if (call == CPG_CALL_ALS_TUNE) {
    for (int c : als_candidates(s, R, &od)) bytes = std::max(bytes, als_bytes(s, R, prec, c, with_copy));
    bytes = als_tune_save_offset(bytes) + als_tune_save_bytes(s, R, prec);
  } else {
    return 0;
  }
  return bytes;
}

}  // namespace

namespace cpg {
size_t workspace_bytes_required(const int64_t* I, int N, int R, const cpg_opts* opts, int call) {
  return workspace_size_impl(I, N, R, opts, call, false);
}

cpg_status gradient_all_arg_status(const void* Y, const int64_t* I, int N, const void* const* A, int R,
                                   void* const* G, const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(A, N) || G == nullptr || !ptrs_ok(const_cast<const void* const*>(G), N))
    return CPG_ERR_ARG;
  return CPG_OK;
}

size_t gradient_all_bytes_for(const int64_t* I, int N, int R, const cpg_opts* opts) {
  Shape s;
  if (opts == nullptr || common_checks(opts, s, I, N, R) != CPG_OK) return 0;
  return grad_bytes(s, R, opts->precision, grad_choice(s, R, opts), false);
}
}  // namespace cpg

extern "C" {

int cpg_split_point(const int64_t* I, int N) {
  Shape s;
  if (check_shape(I, N, 1, s) != CPG_OK) return 0;
  return split_point(s);
}

size_t cpg_workspace_size(const int64_t* I, int N, int R, const cpg_opts* opts, int call) {
  return workspace_size_impl(I, N, R, opts, call, true);
}

cpg_status cp_gradient_all(const void* Y, const int64_t* I, int N, const void* const* A, int R, void* const* G,
                           const cpg_opts* opts) {
  const cpg_status st = cpg::gradient_all_arg_status(Y, I, N, A, R, G, opts);
  if (st != CPG_OK) return st;
  Shape s;
  check_shape(I, N, R, s);
  const GradChoice plan = grad_choice(s, R, opts);
  if (is_f64(opts->precision)) return gradient_all_impl<double>(s, static_cast<const double*>(Y), A, R, G, opts, plan);
  return gradient_all_impl<float>(s, static_cast<const float*>(Y), A, R, G, opts, plan);
}

cpg_status cpg_autotune_gradient(const void* Y, const int64_t* I, int N, const void* const* A, int R, void* const* G,
                                 const cpg_opts* opts, int reps, cpg_gradient_plan* chosen) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(A, N) || G == nullptr || !ptrs_ok(const_cast<const void* const*>(G), N) || reps < 1 ||
      reps > 1000)
    return CPG_ERR_ARG;
  const std::vector<GradChoice> cand = grad_candidates(s, R, opts);
  size_t need = 0;
  for (const GradChoice& c : cand) need = std::max(need, grad_bytes(s, R, opts->precision, c));
  if (opts->workspace == nullptr || opts->workspace_bytes < need) return CPG_ERR_WORKSPACE;
  cudaStream_t str = static_cast<cudaStream_t>(opts->stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CPG_ERR_CUDA;
  auto run = [&](const GradChoice& c) {
    return is_f64(opts->precision)
               ? gradient_all_impl<double>(s, static_cast<const double*>(Y), A, R, G, opts, c)
               : gradient_all_impl<float>(s, static_cast<const float*>(Y), A, R, G, opts, c);
  };
  GradChoice best;
  float best_ms = 0.f;
  bool have = false;
  for (const GradChoice& c : cand) {
    st = run(c);  // first run: planning, attribute setup and warm caches outside the timing
    if (st == CPG_OK && cudaEventRecord(e0, str) != cudaSuccess) st = CPG_ERR_CUDA;
    for (int i = 0; i < reps && st == CPG_OK; ++i) st = run(c);
    if (st == CPG_OK && (cudaEventRecord(e1, str) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      st = CPG_ERR_CUDA;
    if (st != CPG_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= float(reps);
    if (!have || ms < best_ms) {
      best = c;
      best_ms = ms;
      have = true;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CPG_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_tuned[tune_key(s, R, opts)] = best;
  }
  if (chosen) {
    chosen->split = best.k;
    chosen->fused = best.fused ? 1 : 0;
    chosen->ms = best_ms;
    chosen->candidates = int(cand.size());
  }
  return CPG_OK;
}

int cpg_gradient_plan_query(const int64_t* I, int N, int R, const cpg_opts* opts, cpg_gradient_plan* plan) {
  Shape s;
  if (opts == nullptr || check_shape(I, N, R, s) != CPG_OK) return 0;
  GradChoice c;
  if (!tuned_choice(s, R, opts, &c)) return 0;
  if (plan) {
    plan->split = c.k;
    plan->fused = c.fused ? 1 : 0;
    plan->ms = 0.f;
    plan->candidates = 0;
  }
  return 1;
}

cpg_status cpg_gradient_plan_set(const int64_t* I, int N, int R, const cpg_opts* opts, const cpg_gradient_plan* plan) {
  Shape s;
  if (opts == nullptr || plan == nullptr) return CPG_ERR_ARG;
  cpg_status st = check_shape(I, N, R, s);
  if (st != CPG_OK) return st;
  if (!prec_valid(opts->precision)) return CPG_ERR_ARG;
  if (plan->split < 1 || plan->split > N - 1 || (opts->split != 0 && opts->split != plan->split)) return CPG_ERR_ARG;
  GradChoice c;
  c.k = plan->split;
  c.fused = plan->fused != 0;
  if (c.fused && is_tc_prec(opts->precision) && !tc_fused_ok(tc_rank_tile(std::min(R, 64)), tc_code(opts->precision)))
    return CPG_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  g_tuned[tune_key(s, R, opts)] = c;
  return CPG_OK;
}

cpg_status cpg_als_plan_set(const int64_t* I, int N, int R, const cpg_opts* opts, const cpg_als_plan* plan) {
  Shape s;
  if (opts == nullptr || plan == nullptr) return CPG_ERR_ARG;
  cpg_status st = check_shape(I, N, R, s);
  if (st != CPG_OK) return st;
  if (!prec_valid(opts->precision)) return CPG_ERR_ARG;
  if (plan->split < 1 || plan->split > N - 1 || (opts->split != 0 && opts->split != plan->split)) return CPG_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  g_als_tuned[tune_key(s, R, opts)] = plan->split;
  return CPG_OK;
}

void cpg_autotune_clear(void) {
  std::lock_guard<std::mutex> lock(g_tuned_mu);
  g_tuned.clear();
  g_als_tuned.clear();
}

int cpg_als_candidates(const int64_t* I, int N, int R, const cpg_opts* opts, int* splits, int cap) {
  Shape s;
  if (check_shape(I, N, R, s) != CPG_OK || (opts && opts->split != 0 && (opts->split < 1 || opts->split > N - 1)))
    return 0;
  const std::vector<int> c = als_candidates(s, R, opts);
  for (int i = 0; i < int(c.size()) && i < cap && splits; ++i) splits[i] = c[i];
  return int(c.size());
}

cpg_status cpg_autotune_als(const void* Y, const int64_t* I, int N, void* const* A, double* lambda, int R,
                            const cpg_opts* opts, int reps, cpg_als_plan* chosen) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(const_cast<const void* const*>(A), N) || lambda == nullptr || reps < 1 || reps > 1000)
    return CPG_ERR_ARG;
  if (!sweep_prec_ok(opts->precision)) return CPG_ERR_UNSUPPORTED;
  if (R > kAlsMaxRank) return CPG_ERR_UNSUPPORTED;
  const int prec = opts->precision;
  const std::vector<int> cand = als_candidates(s, R, opts);
  size_t als_need = 0;
  for (int k : cand) als_need = std::max(als_need, als_bytes(s, R, prec, k, true));
  const size_t save_off = als_tune_save_offset(als_need);
  if (opts->workspace == nullptr || opts->workspace_bytes < save_off + als_tune_save_bytes(s, R, prec))
    return CPG_ERR_WORKSPACE;
  cudaStream_t str = static_cast<cudaStream_t>(opts->stream);
  const size_t es = is_f64(prec) ? 8 : 4;
  unsigned char* save = static_cast<unsigned char*>(opts->workspace) + save_off;
  // Copies between the caller's factors and lambda and the save area.
  auto copy_all = [&](bool to_save) {
    size_t off = 0;
    for (int n = 0; n < N && st == CPG_OK; ++n) {
      const size_t b = size_t(s.I[n]) * size_t(R) * es;
      void* dst = to_save ? static_cast<void*>(save + off) : A[n];
      const void* src = to_save ? static_cast<const void*>(A[n]) : static_cast<const void*>(save + off);
      if (cudaMemcpyAsync(dst, src, b, cudaMemcpyDeviceToDevice, str) != cudaSuccess) st = CPG_ERR_CUDA;
      off += b;
    }
    off = align_up(off);
    void* dl = to_save ? static_cast<void*>(save + off) : static_cast<void*>(lambda);
    const void* sl = to_save ? static_cast<const void*>(lambda) : static_cast<const void*>(save + off);
    if (st == CPG_OK && cudaMemcpyAsync(dl, sl, size_t(R) * sizeof(double), cudaMemcpyDeviceToDevice, str) != cudaSuccess)
      st = CPG_ERR_CUDA;
  };
  cpg_opts o = *opts;
  o.workspace_bytes = save_off;  // the sweeps never touch the save area
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CPG_ERR_CUDA;
  auto run = [&](int iters) {
    return is_f64(prec) ? als_impl<double>(s, static_cast<const double*>(Y), A, lambda, R, iters, nullptr, &o)
                        : als_impl<float>(s, static_cast<const float*>(Y), A, lambda, R, iters, nullptr, &o);
  };
  copy_all(true);
  int best = 0;
  float best_ms = 0.f;
  for (int k : cand) {
    if (st != CPG_OK) break;
    o.split = k;
    st = run(1);  // untimed: planning, attribute setup and warm caches
    if (st == CPG_ERR_UNSUPPORTED) {  // a split this size cannot run (refused before any launch)
      st = CPG_OK;
      continue;
    }
    copy_all(false);
    if (st == CPG_OK && cudaEventRecord(e0, str) != cudaSuccess) st = CPG_ERR_CUDA;
    if (st == CPG_OK) st = run(reps);
    if (st == CPG_OK && (cudaEventRecord(e1, str) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
      st = CPG_ERR_CUDA;
    copy_all(false);
    if (st != CPG_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= float(reps);
    if (best == 0 || ms < best_ms) {
      best = k;
      best_ms = ms;
    }
  }
  if (cudaStreamSynchronize(str) != cudaSuccess && st == CPG_OK) st = CPG_ERR_CUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != CPG_OK) return st;
  if (best == 0) return CPG_ERR_UNSUPPORTED;  // no candidate could run
  {
    std::lock_guard<std::mutex> lock(g_tuned_mu);
    g_als_tuned[tune_key(s, R, opts)] = best;
  }
  if (chosen) {
    chosen->split = best;
    chosen->ms = best_ms;
    chosen->candidates = int(cand.size());
  }
  return CPG_OK;
}

int cpg_als_plan_query(const int64_t* I, int N, int R, const cpg_opts* opts, cpg_als_plan* plan) {
  Shape s;
  if (opts == nullptr || check_shape(I, N, R, s) != CPG_OK) return 0;
  int k = 0;
  if (!tuned_als_split(s, R, opts, &k)) return 0;
  if (plan) {
    plan->split = k;
    plan->ms = 0.f;
    plan->candidates = 0;
  }
  return 1;
}

cpg_status cp_gradient_mode(const void* Y, const int64_t* I, int N, const void* const* A, int R, int n, void* Gn,
                            const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (n < 0 || n >= N || Y == nullptr || !ptrs_ok(A, N) || Gn == nullptr) return CPG_ERR_ARG;
  if (is_f64(opts->precision))
    return gradient_mode_impl<double>(s, static_cast<const double*>(Y), A, R, n, static_cast<double*>(Gn), opts);
  return gradient_mode_impl<float>(s, static_cast<const float*>(Y), A, R, n, static_cast<float*>(Gn), opts);
}

cpg_status cp_als_iter(const void* Y, const int64_t* I, int N, void* const* A, double* lambda, int R, int iters,
                       double* fit, const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(const_cast<const void* const*>(A), N) || lambda == nullptr || iters < 0)
    return CPG_ERR_ARG;
  if (!sweep_prec_ok(opts->precision)) return CPG_ERR_UNSUPPORTED;
  if (iters == 0) return CPG_OK;
  if (is_f64(opts->precision)) return als_impl<double>(s, static_cast<const double*>(Y), A, lambda, R, iters, fit, opts);
  return als_impl<float>(s, static_cast<const float*>(Y), A, lambda, R, iters, fit, opts);
}

cpg_status cp_gradient_full(const void* Y, const int64_t* I, int N, const void* const* A, int R, void* const* G,
                            const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(A, N) || G == nullptr || !ptrs_ok(const_cast<const void* const*>(G), N))
    return CPG_ERR_ARG;
  void* const* Am = const_cast<void* const*>(A);  // read only: no step
  if (is_f64(opts->precision))
    return gradient_full_impl<double>(s, static_cast<const double*>(Y), Am, R, G, opts, 0.0, false);
  return gradient_full_impl<float>(s, static_cast<const float*>(Y), Am, R, G, opts, 0.0, false);
}

cpg_status cp_gradient_step(const void* Y, const int64_t* I, int N, void* const* A, int R, double eta, void* const* G,
                            const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(const_cast<const void* const*>(A), N) || G == nullptr ||
      !ptrs_ok(const_cast<const void* const*>(G), N) || !(eta == eta))
    return CPG_ERR_ARG;
  if (is_f64(opts->precision))
    return gradient_full_impl<double>(s, static_cast<const double*>(Y), A, R, G, opts, eta, true);
  return gradient_full_impl<float>(s, static_cast<const float*>(Y), A, R, G, opts, eta, true);
}

cpg_status cp_ntf_iter(const void* Y, const int64_t* I, int N, void* const* A, int R, int iters, double* fit,
                       const cpg_opts* opts) {
  Shape s;
  cpg_status st = common_checks(opts, s, I, N, R);
  if (st != CPG_OK) return st;
  if (Y == nullptr || !ptrs_ok(const_cast<const void* const*>(A), N) || iters < 0) return CPG_ERR_ARG;
  if (!sweep_prec_ok(opts->precision)) return CPG_ERR_UNSUPPORTED;
  if (iters == 0) return CPG_OK;
  if (is_f64(opts->precision))
    return als_impl<double>(s, static_cast<const double*>(Y), A, nullptr, R, iters, fit, opts, nullptr, true);
  return als_impl<float>(s, static_cast<const float*>(Y), A, nullptr, R, iters, fit, opts, nullptr, true);
}

cpg_status cpg_selftest_timeout(const cpg_opts* opts, unsigned polls) {
  if (opts == nullptr || opts->workspace == nullptr || opts->workspace_bytes < kAlign || polls < 1 ||
      polls > (1u << 24))
    return CPG_ERR_ARG;
  ++g_launches;
  timeout_selftest_kernel<<<1, 32, 0, static_cast<cudaStream_t>(opts->stream)>>>(static_cast<int*>(opts->workspace),
                                                                                 polls);
  return cuda_status(cudaGetLastError());
}

cpg_status cpg_workspace_init(const cpg_opts* opts) {
  if (opts == nullptr || opts->workspace == nullptr || opts->workspace_bytes < kAlign) return CPG_ERR_ARG;
  ++g_launches;
  return cuda_status(cudaMemsetAsync(opts->workspace, 0, kAlign, static_cast<cudaStream_t>(opts->stream)));
}

cpg_status cpg_device_status(const cpg_opts* opts) {
  if (opts == nullptr || opts->workspace == nullptr) return CPG_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(opts->stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return CPG_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, opts->workspace, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CPG_ERR_CUDA;
  const int zero = 0;
  if (cudaMemcpy(opts->workspace, &zero, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return CPG_ERR_CUDA;
  return static_cast<cpg_status>(v);
}

const char* cpg_status_str(int status) {
  switch (status) {
    case CPG_OK: return "ok";
    case CPG_ERR_ARG: return "invalid argument";
    case CPG_ERR_SHAPE: return "tensor size overflows int64";
    case CPG_ERR_WORKSPACE: return "workspace missing or too small";
    case CPG_ERR_SINGULAR: return "normal-equation matrix not positive definite";
    case CPG_ERR_CUDA: return "CUDA launch or runtime error";
    case CPG_ERR_TIMEOUT: return "bounded device wait expired";
    case CPG_ERR_UNSUPPORTED: return "unsupported precision or size for this call";
    default: return "unknown status";
  }
}

int cpg_profile_lead(int enable) {
  if (enable && !g_timing.made) {
    for (int i = 0; i < 2 * LeadTiming::kMax; ++i)
      if (cudaEventCreate(&g_timing.ev[i]) != cudaSuccess) return CPG_ERR_CUDA;
    g_timing.made = true;
  }
  g_timing.on = enable != 0;
  g_timing.all = enable == 2;
  g_timing.n = 0;
  return CPG_OK;
}

int cpg_profile_read(float* ms, int* sides, int max) {
  if (!g_timing.made) return 0;
  const int n = std::min(g_timing.n, max);
  for (int i = 0; i < n; ++i) {
    if (cudaEventSynchronize(g_timing.ev[2 * i + 1]) != cudaSuccess) return -1;
    float t = 0.f;
    cudaEventElapsedTime(&t, g_timing.ev[2 * i], g_timing.ev[2 * i + 1]);
    if (ms) ms[i] = t;
    if (sides) sides[i] = g_timing.sides[i];
  }
  g_timing.n = 0;
  return n;
}

size_t cpg_workspace_size_batched(int B, const cpg_tensor_desc* descs, const cpg_opts* opts) {
  if (B < 1 || descs == nullptr) return 0;
  size_t total = kAlign;  // the shared status word
  for (int b = 0; b < B; ++b) {
    const size_t m = member_ws_bytes(descs[b], opts);
    if (m == 0) return 0;
    total += align_up(m);
  }
  return total;
}

cpg_status cp_als_batched(int B, const cpg_tensor_desc* descs, int iters, const cpg_opts* opts) {
  if (opts == nullptr || B < 1 || descs == nullptr || iters < 0) return CPG_ERR_ARG;
  if (!prec_valid(opts->precision)) return CPG_ERR_ARG;
  if (!sweep_prec_ok(opts->precision)) return CPG_ERR_UNSUPPORTED;
  // Validate every member before launching anything.
  std::vector<Shape> shapes(B);
  std::vector<size_t> off(B);
  size_t total = kAlign;
  for (int b = 0; b < B; ++b) {
    const cpg_tensor_desc& d = descs[b];
    cpg_status st = check_shape(d.I, d.N, d.R, shapes[b]);
    if (st != CPG_OK) return st;
    if (opts->split != 0 && (opts->split < 1 || opts->split > d.N - 1)) return CPG_ERR_ARG;
    if (d.Y == nullptr || !ptrs_ok(const_cast<const void* const*>(d.A), d.N) || d.lambda == nullptr)
      return CPG_ERR_ARG;
    if (d.R > kAlsMaxRank) return CPG_ERR_UNSUPPORTED;
    const size_t m = member_ws_bytes(d, opts);
    if (m == 0) return CPG_ERR_ARG;
    off[b] = total;
    total += align_up(m);
  }
  if (opts->workspace == nullptr || opts->workspace_bytes < total) return CPG_ERR_WORKSPACE;
  if (iters == 0) return CPG_OK;
  StreamPool* pool = stream_pool();
  if (pool == nullptr) return CPG_ERR_CUDA;
  cudaStream_t caller = static_cast<cudaStream_t>(opts->stream);
  int* status = static_cast<int*>(opts->workspace);

  // Largest members first, each to the stream with the least work so far
  // (work ~ tensor entries x max(R, 8) per sweep plus a fixed chain cost).
  std::vector<int> ord(B);
  for (int b = 0; b < B; ++b) ord[b] = b;
  auto work = [&](int b) { return double(shapes[b].total) * std::max(descs[b].R, 8) + 2e6 * shapes[b].N; };
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return work(x) > work(y); });
  const int ns = std::min(B, kPoolStreams);
  std::vector<double> load(ns, 0.0);
  std::vector<int> used(ns, 0);
  if (cudaEventRecord(pool->fork, caller) != cudaSuccess) return CPG_ERR_CUDA;
  cpg_status result = CPG_OK;
  for (int b : ord) {
    const int i = int(std::min_element(load.begin(), load.end()) - load.begin());
    load[i] += work(b);
    if (!used[i]) {
      if (cudaStreamWaitEvent(pool->s[i], pool->fork, 0) != cudaSuccess) return CPG_ERR_CUDA;
      used[i] = 1;
    }
    const cpg_tensor_desc& d = descs[b];
    cpg_opts mo = *opts;
    mo.workspace = static_cast<char*>(opts->workspace) + off[b];
    mo.workspace_bytes = total - off[b];
    mo.stream = pool->s[i];
    const cpg_status st =
        is_f64(opts->precision)
            ? als_impl<double>(shapes[b], static_cast<const double*>(d.Y), d.A, d.lambda, d.R, iters, d.fit, &mo,
                               status)
            : als_impl<float>(shapes[b], static_cast<const float*>(d.Y), d.A, d.lambda, d.R, iters, d.fit, &mo, status);
    if (st != CPG_OK) {
      result = st;
      break;
    }
  }
  // Join every stream that was forked, whatever happened above.
  for (int i = 0; i < ns; ++i) {
    if (!used[i]) continue;
    if (cudaEventRecord(pool->join[i], pool->s[i]) != cudaSuccess ||
        cudaStreamWaitEvent(caller, pool->join[i], 0) != cudaSuccess)
      result = CPG_ERR_CUDA;
  }
  return result;
}

uint64_t cpg_launch_count(int reset) {
  const uint64_t v = g_launches;
  if (reset) g_launches = 0;
  return v;
}

}  // extern "C"
