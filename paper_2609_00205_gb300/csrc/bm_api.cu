// C ABI of the BlockMGARD GPU library: argument checks, plans, scratch,
// stream layout and the order of the kernels of each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/blockmgard.h"
#include "bm_adjoint.cuh"
#include "bm_global.cuh"
#include "bm_huffman.cuh"
#include "bm_internal.h"
#include "bm_plan.h"
#include "bm_qtab.cuh"

#ifndef BM_FWD_HIST
#define BM_FWD_HIST 0
#endif
// The block region's histogram: on a second stream beside the global levels
// (BM_HIST_OVERLAP) with BM_HIST_CTAS CTAs per SM.
// BM_CB_PRESORT: a compress call's codebook starts with the multi-CTA
// clearing, compaction and sort of cb_presort_kernel and, above 8192 present
// symbols, ends with the multi-CTA emission of cb_emit_kernel.
#ifndef BM_CB_PRESORT
#define BM_CB_PRESORT 1
#endif
// BM_BATCH_GRAPHS: a batched compress met a second time with the same
// arguments is captured as a CUDA graph, and replayed from then on.
#ifndef BM_BATCH_GRAPHS
#define BM_BATCH_GRAPHS 1
#endif
// Percentage of the SMs the block symbols' wide-window histogram takes (the
// rest run the global levels beside it: one of its CTAs holds most of an SM's
// shared memory, so on every SM it takes, the global levels' kernels wait).
// On GB300 at 513^3 a compress call took 1.276 / 1.526 / 2.384 / 2.848 ms
// (1e-2 .. 1e-5) with 66 against 1.335 / 1.577 / 2.432 / 2.934 with 100,
// 1.316 / 1.556 / 2.419 / 2.932 with 50 and 1.320 / 1.560 / 2.426 / 2.883
// with 80.
#ifndef BM_HIST_WIDE_PCT
#define BM_HIST_WIDE_PCT 66
#endif
#ifndef BM_HIST_OVERLAP
#define BM_HIST_OVERLAP 1
#endif
#ifndef BM_HIST_CTAS
#define BM_HIST_CTAS 2
#endif

namespace bm {
namespace {

// ---------------------------------------------------------------------------
// Errors, counters, timing
// ---------------------------------------------------------------------------
thread_local std::string g_detail;
std::atomic<uint64_t> g_launches{0};
std::atomic<int> g_timing{0};
// bumped whenever library scratch is (re)allocated: captured batch graphs
// holding older addresses are discarded
std::atomic<uint64_t> g_alloc_gen{0};

struct StageTimer {
  struct Rec { const char* name; cudaEvent_t a, b; cudaStream_t s; };
  std::vector<Rec> recs;
  struct Done { const char* name; float ms, start; };
  std::vector<Done> last;
  cudaStream_t s = nullptr;
  bool on = false;
  void begin(cudaStream_t st) {
    clear();
    s = st;
    on = g_timing.load() != 0;
  }
  std::vector<std::pair<int, cudaEvent_t>> pool;  // (device, event), reused across calls
  cudaEvent_t take() {
    int dev = 0;
    cudaGetDevice(&dev);
    for (size_t i = pool.size(); i-- > 0;)
      if (pool[i].first == dev) {
        cudaEvent_t e = pool[i].second;
        pool.erase(pool.begin() + (long)i);
        return e;
      }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void clear() {
    int dev = 0;
    cudaGetDevice(&dev);
    for (auto& r : recs) { pool.push_back({dev, r.a}); pool.push_back({dev, r.b}); }
    recs.clear();
  }
  int open(const char* name, cudaStream_t st) {
    if (!on) return -1;
    Rec r{name, take(), take(), st ? st : s};
    cudaEventRecord(r.a, r.s);
    recs.push_back(r);
    return (int)recs.size() - 1;
  }
  void close(int i) {
    if (i >= 0) cudaEventRecord(recs[i].b, recs[i].s);
  }
  void collect() {
    if (!on) return;
    last.clear();
    for (auto& r : recs) {
      float ms = 0.f, t0 = 0.f;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&ms, r.a, r.b);
      cudaEventElapsedTime(&t0, recs[0].a, r.a);
      last.push_back({r.name, ms, t0});
    }
    clear();
  }
};
std::mutex g_timer_mu;
StageTimer g_timer;

struct Stage {  // times a stage on the call's stream (or on `st`)
  int i;
  explicit Stage(const char* n, cudaStream_t st = nullptr) : i(g_timer.open(n, st)) {}
  ~Stage() { g_timer.close(i); }
};

bm_status fail(bm_status s, const std::string& msg) {
  g_detail = msg;
  return s;
}

#define BM_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail(BM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define BM_LAUNCHED() g_launches.fetch_add(1)

int num_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  static std::mutex mu;
  static std::map<int, int> cache;
  std::lock_guard<std::mutex> g(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  cache[dev] = n > 0 ? n : 1;
  return cache[dev];
}

// ---------------------------------------------------------------------------
// Scratch: one grow-only device buffer (+ pinned host buffer) per stream
// ---------------------------------------------------------------------------
struct Workspace {
  void* d = nullptr;
  size_t dbytes = 0;
  void* h = nullptr;
  void* hd = nullptr;  // device-side address of h (pinned memory is mapped)
  size_t hbytes = 0;
  int dev = -1;
  // second stream for work that runs beside the caller's stream, joined back
  // into it by an event before the call returns
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

bm_status ensure_aux(Workspace* w) {
  if (w->aux) return BM_OK;
  BM_CUDA(cudaStreamCreateWithFlags(&w->aux, cudaStreamNonBlocking));
  BM_CUDA(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
  BM_CUDA(cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming));
  return BM_OK;
}
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

bm_status get_ws(cudaStream_t s, size_t dbytes, size_t hbytes, Workspace** out) {
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(g_ws_mu);
  Workspace& w = g_ws[{dev, s}];
  w.dev = dev;
  if (w.dbytes < dbytes) {
    if (w.d) { cudaStreamSynchronize(s); cudaFree(w.d); w.d = nullptr; w.dbytes = 0; }
    size_t want = dbytes + dbytes / 8 + (1 << 20);
    g_alloc_gen.fetch_add(1);
    if (cudaMalloc(&w.d, want) != cudaSuccess) {
      cudaGetLastError();
      w.d = nullptr;
      return fail(BM_ERR_OOM, "cudaMalloc of " + std::to_string(want) + " scratch bytes failed");
    }
    w.dbytes = want;
  }
  if (w.hbytes < hbytes) {
    if (w.h) { cudaStreamSynchronize(s); cudaFreeHost(w.h); w.h = nullptr; w.hd = nullptr; w.hbytes = 0; }
    size_t want = hbytes + (1 << 16);
    g_alloc_gen.fetch_add(1);
    if (cudaMallocHost(&w.h, want) != cudaSuccess) {
      cudaGetLastError();
      w.h = nullptr;
      return fail(BM_ERR_OOM, "pinned host scratch allocation failed");
    }
    if (cudaHostGetDevicePointer(&w.hd, w.h, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(w.h);
      w.h = nullptr;
      w.hd = nullptr;
      return fail(BM_ERR_CUDA, "pinned host scratch is not mapped into the device address space");
    }
    w.hbytes = want;
  }
  *out = &w;
  return BM_OK;
}

// Sequential sub-allocation of a scratch buffer, 256-byte aligned.
struct Carver {
  size_t off = 0;
  unsigned char* base = nullptr;
  template <typename X>
  X* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    X* p = reinterpret_cast<X*>(base ? base + off : nullptr);
    off += count * sizeof(X);
    return p;
  }
};

// ---------------------------------------------------------------------------
// Plans (host tables + device copies of the global-level tables)
// ---------------------------------------------------------------------------
struct PlanDev {
  PlanHost h;
  void* dtab[2] = {nullptr, nullptr};  // per dtype
  int dev[2] = {-1, -1};
  std::vector<GLevel<float>> gf;
  std::vector<GLevel<double>> gd;
  std::vector<GLevel<float>> rf;   // in-cache levels on the block-major grid (fields with an extent of 1)
  std::vector<GLevel<double>> rd;
  std::vector<std::vector<GLevel<float>>> xf;   // [round][level] blocked levels (no fused block kernel)
  std::vector<std::vector<GLevel<double>>> xd;
};
std::mutex g_plan_mu;
std::map<std::tuple<int64_t, int64_t, int64_t, int, int, int, int>, std::unique_ptr<PlanDev>> g_plans;

template <typename T>
std::vector<GLevel<T>>& glevels(PlanDev& p);
template <>
std::vector<GLevel<float>>& glevels<float>(PlanDev& p) { return p.gf; }
template <>
std::vector<GLevel<double>>& glevels<double>(PlanDev& p) { return p.gd; }
template <typename T>
std::vector<std::vector<GLevel<T>>>& xlevels(PlanDev& p);
template <>
std::vector<std::vector<GLevel<float>>>& xlevels<float>(PlanDev& p) { return p.xf; }
template <>
std::vector<std::vector<GLevel<double>>>& xlevels<double>(PlanDev& p) { return p.xd; }
template <typename T>
std::vector<GLevel<T>>& rlevels(PlanDev& p);
template <>
std::vector<GLevel<float>>& rlevels<float>(PlanDev& p) { return p.rf; }
template <>
std::vector<GLevel<double>>& rlevels<double>(PlanDev& p) { return p.rd; }

template <typename T>
bm_status upload_tables(PlanDev& P) {
  const int di = sizeof(T) == 8 ? 1 : 0;
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  if (P.dtab[di] && P.dev[di] == dev) return BM_OK;
  // host image: per level per dim the arrays in a fixed order
  std::vector<unsigned char> img;
  auto put = [&](const void* src, size_t bytes) {
    size_t off = (img.size() + 15) & ~size_t(15);
    img.resize(off + bytes);
    if (bytes) std::memcpy(img.data() + off, src, bytes);
    return off;
  };
  struct Offs { size_t cidx, jlo, jhi, wl, wr, cb, isc, proj, f0, band, tm, tib, tsup, md, mo; };
  std::vector<Offs> offs;
  // every tabulated dimension: the global levels' three, then the two in-block
  // axes of each in-cache level of the block-major grid
  std::vector<const Dim1DHost*> dims;
  for (auto& L3 : P.h.glev)
    for (auto& D : L3) dims.push_back(&D);
  for (auto& rl : P.h.rlev) {
    dims.push_back(&rl.da);
    dims.push_back(&rl.db);
  }
  for (auto& rlv : P.h.xlev)
    for (auto& X : rlv)
      for (int d = 0; d < 3; ++d) dims.push_back(&X.d[d]);
  for (const Dim1DHost* Dp : dims) {
    const Dim1DHost& D = *Dp;
    {
      auto cvt = [](const std::vector<double>& v) {
        std::vector<T> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = (T)v[i];
        return o;
      };
      std::vector<T> wl = cvt(D.wl), wr = cvt(D.wr), proj = cvt(D.P), band = cvt(D.band), tm = cvt(D.tm),
                     tib = cvt(D.tib), tsup = cvt(D.tsup), md = cvt(D.md), mo = cvt(D.mo);
      Offs o;
      o.cidx = put(D.cidx.data(), D.cidx.size() * 4);
      o.jlo = put(D.jlo.data(), D.jlo.size() * 4);
      o.jhi = put(D.jhi.data(), D.jhi.size() * 4);
      o.wl = put(wl.data(), wl.size() * sizeof(T));
      o.wr = put(wr.data(), wr.size() * sizeof(T));
      o.cb = put(D.cb.data(), D.cb.size() * 4);
      o.isc = put(D.isc.data(), D.isc.size());
      o.proj = put(proj.data(), proj.size() * sizeof(T));
      o.f0 = put(D.f0.data(), D.f0.size() * 4);
      o.band = put(band.data(), band.size() * sizeof(T));
      o.tm = put(tm.data(), tm.size() * sizeof(T));
      o.tib = put(tib.data(), tib.size() * sizeof(T));
      o.tsup = put(tsup.data(), tsup.size() * sizeof(T));
      o.md = put(md.data(), md.size() * sizeof(T));
      o.mo = put(mo.data(), mo.size() * sizeof(T));
      offs.push_back(o);
    }
  }
  if (P.dtab[di]) { cudaFree(P.dtab[di]); P.dtab[di] = nullptr; }
  if (!img.empty()) {
    BM_CUDA(cudaMalloc(&P.dtab[di], img.size()));
    BM_CUDA(cudaMemcpy(P.dtab[di], img.data(), img.size(), cudaMemcpyHostToDevice));
  }
  P.dev[di] = dev;
  auto& G = glevels<T>(P);
  G.clear();
  const unsigned char* base = reinterpret_cast<const unsigned char*>(P.dtab[di]);
  auto fill = [&](GDim<T>& g, const Offs& o, const Dim1DHost& D) {
    {
      g.n = D.n; g.c = D.c;
      g.cidx = reinterpret_cast<const int*>(base + o.cidx);
      g.jlo = reinterpret_cast<const int*>(base + o.jlo);
      g.jhi = reinterpret_cast<const int*>(base + o.jhi);
      g.wl = reinterpret_cast<const T*>(base + o.wl);
      g.wr = reinterpret_cast<const T*>(base + o.wr);
      g.cb = reinterpret_cast<const int*>(base + o.cb);
      g.isc = reinterpret_cast<const uint8_t*>(base + o.isc);
      g.P = reinterpret_cast<const T*>(base + o.proj);
      g.f0 = reinterpret_cast<const int*>(base + o.f0);
      g.band = reinterpret_cast<const T*>(base + o.band);
      g.tm = reinterpret_cast<const T*>(base + o.tm);
      g.tib = reinterpret_cast<const T*>(base + o.tib);
      g.tsup = reinterpret_cast<const T*>(base + o.tsup);
      g.md = reinterpret_cast<const T*>(base + o.md);
      g.mo = reinterpret_cast<const T*>(base + o.mo);
      g.ident = 0;
    }
  };
  for (int l = 0; l < P.h.M; ++l) {
    GLevel<T> L{};
    for (int d = 0; d < 3; ++d) fill(L.d[d], offs[(size_t)(l * 3 + d)], P.h.glev[l][d]);
    L.sym_off = P.h.sym_off[l];
    L.blk_extra = 0;
    G.push_back(L);
  }
  auto& RL = rlevels<T>(P);
  RL.clear();
  size_t k = (size_t)P.h.M * 3;
  for (const RLevelHost& rl : P.h.rlev) {
    GLevel<T> L{};
    L.d[0].n = L.d[0].c = (int)rl.nblk;
    L.d[0].ident = 1;
    fill(L.d[1], offs[k], rl.da);
    fill(L.d[2], offs[k + 1], rl.db);
    k += 2;
    L.sym_off = rl.off;
    L.blk_extra = rl.blk_extra;
    RL.push_back(L);
  }
  auto& XL = xlevels<T>(P);
  XL.clear();
  for (auto& rlv : P.h.xlev) {
    std::vector<GLevel<T>> lv;
    for (auto& X : rlv) {
      GLevel<T> L{};
      for (int d = 0; d < 3; ++d) {
        fill(L.d[d], offs[k++], X.d[d]);
        L.be[d] = X.e[d];
        L.bce[d] = X.ce[d];
        L.bnb[d] = X.nb[d];
      }
      L.sym_off = X.sym_off;
      L.blk_extra = 0;
      L.bmode = 1;
      L.bpb = P.h.per_block;
      lv.push_back(L);
    }
    XL.push_back(lv);
  }
  return BM_OK;
}

bm_status get_plan(const int64_t* shape, int B, int K, int M, int R, PlanDev** out) {
  std::lock_guard<std::mutex> g(g_plan_mu);
  auto key = std::make_tuple(shape[0], shape[1], shape[2], B, K, M, R);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    auto p = std::make_unique<PlanDev>();
    std::string err = make_plan(shape, B, K, M, R, p->h);
    if (!err.empty()) return fail(BM_ERR_ARG, err);
    it = g_plans.emplace(key, std::move(p)).first;
  }
  *out = it->second.get();
  return BM_OK;
}

// ---------------------------------------------------------------------------
// Parameters and shapes
// ---------------------------------------------------------------------------
struct Params { int B, K, M, chunk, radius, R, ndim = 3; };

bm_status check_params(const bm_params* p, Params& o) {
  o.B = (p && p->block_nodes) ? p->block_nodes : 17;
  o.K = (p && p->incache_levels) ? p->incache_levels : 2;
  o.M = (p && p->global_levels) ? p->global_levels : 2;
  if (p && p->global_levels < 0) o.M = 0;
  o.chunk = (p && p->chunk_symbols) ? p->chunk_symbols : 2048;
  o.radius = (p && p->dict_radius) ? p->dict_radius : kMaxDict / 2;
  o.R = (p && p->rounds) ? p->rounds : 1;
  if (o.R < 1 || o.R > 8) return fail(BM_ERR_ARG, "rounds must be in [1, 8]");
  if (o.B < 3 || o.B > 64) return fail(BM_ERR_ARG, "block_nodes must be in [3, 64]");
  int kmax = 0;  // levels while a block edge still has at least 3 nodes
  for (int n = o.B; n >= 3; n = n / 2 + 1) ++kmax;
  if (o.K < 1 || o.K > kmax) return fail(BM_ERR_ARG, "incache_levels out of range for this block size");
  if (o.M > 16) return fail(BM_ERR_ARG, "global_levels too large");
  if (o.chunk < 64 || o.chunk > 2048 || o.chunk % 32) return fail(BM_ERR_ARG, "chunk_symbols must be a multiple of 32 in [64, 2048]");
  if (o.radius < 16 || o.radius > kMaxDict / 2) return fail(BM_ERR_ARG, "dict_radius must be in [16, 32768]");
  return BM_OK;
}

// A field of ndim (1..3) dimensions as a 3-D shape with leading extents of 1
// (a dimension of extent 1 is neither blocked nor coarsened); at least two
// values.
bm_status norm_shape(int ndim, const int64_t* shape, int64_t s3[3]) {
  if (ndim < 1 || ndim > 3) return fail(BM_ERR_ARG, "ndim must be 1, 2 or 3");
  if (!shape) return fail(BM_ERR_ARG, "shape is NULL");
  int64_t total = 1;
  for (int d = 0; d < 3; ++d) {
    s3[d] = d < 3 - ndim ? 1 : shape[d - (3 - ndim)];
    if (s3[d] < 1 || s3[d] > (int64_t(1) << 31)) return fail(BM_ERR_ARG, "every extent must be in [1, 2^31]");
    total *= s3[d];
  }
  if (total < 2) return fail(BM_ERR_ARG, "a field needs at least two values");
  return BM_OK;
}

int64_t nel3(const int64_t* s) { return s[0] * s[1] * s[2]; }

// Sizes of the global-level scratch arrays (elements): U[l] per level, D, W1,
// W2; for a field with an extent of 1, RB[l] (l = 0..K) the block-major grids
// of its in-cache levels (the same D, W1, W2 serve their passes).
struct GSizes {
  std::vector<int64_t> U;
  int64_t D = 0, W1 = 0, W2 = 0;
  std::vector<int64_t> RB;
  std::vector<int64_t> XP;  // padded grids of the blocked levels 0..K-1 (no fused block kernel)
};
GSizes gsizes(const PlanHost& h) {
  GSizes g;
  for (int l = 0; l <= h.M; ++l) g.U.push_back(h.lshape[3 * l] * h.lshape[3 * l + 1] * h.lshape[3 * l + 2]);
  g.D = g.U[0];
  for (int l = 0; l < h.M; ++l) {
    const int64_t n0 = h.lshape[3 * l], n1 = h.lshape[3 * l + 1];
    const int64_t c0 = h.lshape[3 * l + 3], c1 = h.lshape[3 * l + 4], c2 = h.lshape[3 * l + 5];
    g.W1 = std::max(g.W1, n0 * n1 * c2);
    g.W2 = std::max(g.W2, std::max(n0 * c1 * c2, c0 * c1 * c2));
  }
  if (h.generic) {  // padded grids of every level, sized for the largest round
    for (int l = 0; l < h.K; ++l) {
      int64_t big = 0;
      for (const auto& rlv : h.xlev) {
        const XLevelHost& X = rlv[(size_t)l];
        const int64_t n0 = X.shape[0], n1 = X.shape[1], n2 = X.shape[2];
        const int64_t c0 = X.d[0].c, c1 = X.d[1].c, c2 = X.d[2].c;
        big = std::max(big, n0 * n1 * n2);
        g.W1 = std::max(g.W1, n0 * n1 * c2);
        g.W2 = std::max(g.W2, std::max(n0 * c1 * c2, c0 * c1 * c2));
      }
      g.XP.push_back(big);
      g.D = std::max(g.D, big);
    }
  }
  if (h.reduced) {
    for (const RLevelHost& rl : h.rlev) {
      g.RB.push_back(rl.nblk * rl.da.n * rl.db.n);
      g.W1 = std::max(g.W1, rl.nblk * rl.da.n * rl.db.c);
      g.W2 = std::max(g.W2, rl.nblk * rl.da.c * rl.db.c);
    }
    const RLevelHost& last = h.rlev.back();
    g.RB.push_back(last.nblk * last.da.c * last.db.c);
    g.D = std::max(g.D, g.RB[0]);
  }
  return g;
}

// Between a grid and its block-major tiles (reblock_kernel): the field and
// the blocks of round 0, or the gathered grid G and the blocks' coarse values.
Reblock reblock_of(const PlanHost& h, bool coarse) {
  Reblock R{};
  for (int d = 0; d < 3; ++d) {
    R.g[d] = coarse ? h.gshape[d] : h.shape[d];
    R.e[d] = coarse ? h.md[d] : h.Bd[d];
    R.nb[d] = h.nb[d];
  }
  R.ax[0] = h.ax[0];
  R.ax[1] = h.ax[1];
  const int edge = coarse ? h.m : h.B;
  R.E1 = h.ax[0] < 0 ? 1 : edge;
  R.E2 = edge;
  R.nblk = h.nblocks;
  return R;
}

// cudaFuncAttributeMaxDynamicSharedMemorySize set once per device for a kernel.
std::atomic<unsigned> g_cb_attr{0}, g_dt_attr{0}, g_dec_attr{0}, g_encw_attr{0}, g_encc_attr{0}, g_cbb_attr{0};
std::atomic<unsigned> g_enc1_attr{0}, g_enc3_attr{0};
template <class F>
cudaError_t set_smem_once(F* fn, int bytes, std::atomic<unsigned>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = 1u << (dev & 31);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

// Preferred shared-memory carveout 0 (the most L1) for a kernel that keeps
// a table in L1 rather than in shared memory, once per device.
template <class F>
cudaError_t prefer_l1_once(F* fn, std::atomic<unsigned>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned bit = 1u << (dev & 31);
  if (done.load() & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

int grid_for(int64_t work, int threads, int per_sm = 8) {
  int64_t g = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)num_sms() * per_sm;
  if (g > cap) g = cap;
  return (int)std::max<int64_t>(g, 1);
}

// CTAs of the decoder an SM holds (its lookup table, threads and registers),
// once per device.
int dec_per_sm() {
  static std::atomic<int> cached[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return 1;
  int v = cached[dev].load();
  if (v <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, decode_kernel, kDecThreads, kDecSmem) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    cached[dev].store(v);
  }
  return v;
}

// Histogram of symbols [s0, s1) into hist (zeroed by the caller): with
// `ctas` CTAs of the small-window kernel when the dictionary fits its window,
// else one wide-window CTA per SM (at most `ctas`).  With `check`, symbols
// not below dict are flagged in sc.
std::atomic<unsigned> g_hw_attr{0};
cudaError_t launch_hist(const uint16_t* sym, unsigned long long s0, unsigned long long s1, int dict, unsigned centre,
                        unsigned* hist, Scalars* sc, bool check, int ctas, cudaStream_t s) {
  if (dict <= kHistWin) {
    if (check) hist_kernel<<<ctas, 256, 0, s>>>(sym + s0, s1 - s0, dict, hist, sc);
    else hist_range_kernel<<<ctas, 256, 0, s>>>(sym, s0, s1, dict, centre, hist);
  } else {
    const int smem = 4 * hist_wide_bins(dict);
    const cudaError_t e = set_smem_once(hist_wide_kernel, 4 * kHistWideMax, g_hw_attr);
    if (e != cudaSuccess) return e;
    const int grid = std::max(1, std::min(ctas, num_sms()));
    hist_wide_kernel<<<grid, kHistWideThreads, smem, s>>>(sym, s0, s1, dict, centre, hist, check ? sc : nullptr);
  }
  g_launches.fetch_add(1);
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// Small kernels of the API layer
// ---------------------------------------------------------------------------
// Loads in flight per thread and CTAs per SM of the max|u| pass (the fastest
// measured on GB300 at 513^3 FP32: 0.101 ms, against 0.115 ms with 4 and 8).
#ifndef BM_MAXABS_INFLIGHT
#define BM_MAXABS_INFLIGHT 8
#endif
#ifndef BM_MAXABS_CTAS
#define BM_MAXABS_CTAS 16
#endif

// max |u| (NaN ignored, non-finite values flagged), 16-byte loads over the
// aligned bulk of the field.  The last CTA to finish computes the quantiser
// table from it (qtab_compute) when qa.enabled.
template <typename T>
__global__ void __launch_bounds__(256) maxabs_kernel(const T* __restrict__ u, int64_t n, Scalars* sc, QtabArgs qa) {
  __shared__ bool s_last;
  T m = T(0);
  bool bad = false;
  constexpr int V = 16 / sizeof(T);
  const int64_t head = (int64_t)((16 - (reinterpret_cast<uintptr_t>(u) & 15)) & 15) / (int64_t)sizeof(T);
  const int64_t h = head < n ? head : n;
  const int64_t nv = (n - h) / V;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const uint4* pv = reinterpret_cast<const uint4*>(u + h);
  int64_t i = tid;
  constexpr int NF = BM_MAXABS_INFLIGHT;
  for (; i + (NF - 1) * nth < nv; i += NF * nth) {  // NF 16-byte loads in flight
    uint4 q[NF];
#pragma unroll
    for (int r = 0; r < NF; ++r) q[r] = __ldg(pv + i + r * nth);
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      const T* t = reinterpret_cast<const T*>(&q[r]);
#pragma unroll
      for (int j = 0; j < V; ++j) maxabs_acc(t[j], m, bad);
    }
  }
  for (; i < nv; i += nth) {
    const uint4 q = __ldg(pv + i);
    const T* t = reinterpret_cast<const T*>(&q);
#pragma unroll
    for (int j = 0; j < V; ++j) maxabs_acc(t[j], m, bad);
  }
  for (int64_t i = tid; i < h; i += nth) maxabs_acc(u[i], m, bad);
  for (int64_t i = h + nv * V + tid; i < n; i += nth) maxabs_acc(u[i], m, bad);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const T y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y > m ? y : m;
  }
  bad = __any_sync(0xffffffffu, bad);
  // one atomic per CTA: the whole grid's atomics go to one address
  __shared__ T s_m[8];
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    s_m[threadIdx.x >> 5] = m;
    if (bad) s_bad = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = s_m[w] > m ? s_m[w] : m;
    if (sizeof(T) == 4) atomicMax(&sc->maxabs_bits, (unsigned long long)__float_as_uint((float)m));
    else atomicMax(&sc->maxabs_bits, (unsigned long long)__double_as_longlong((double)m));
    if (s_bad) atomicOr(&sc->status, ST_RAW);
  }
  if (!qa.enabled) return;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&sc->maxabs_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    qtab_compute(qa);
  }
}

struct HeaderArgs {
  uint8_t* out;
  int f64, B, K, M, chunk, radius, ntiers, m, rel, R, ndim;
  int64_t shape[3];
  int nb[3];
  double tol;
  unsigned long long n_symbols, n_chunks, off_tiers, off_qtab, off_btier, off_chunks, off_splits, off_codebook;
  unsigned long long raw_total, capacity;
  Scalars* sc;
};

template <typename V>
__device__ __forceinline__ void put(uint8_t* p, size_t off, V v) { *reinterpret_cast<V*>(p + off) = v; }

// Header of a coded stream; also zeroes the padding after the bitstream and
// the outlier section.
__global__ void header_kernel(HeaderArgs a) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Scalars* sc = a.sc;
  encode_finish(a.raw_total, a.capacity, sc);
  if (sc->status & ST_RAW) return;
  uint8_t* o = a.out;
  put<uint32_t>(o, 0, kMagic);
  put<uint16_t>(o, 4, 1);
  put<uint16_t>(o, 6, (uint16_t)(a.f64 ? 2 : 0));
  put<int32_t>(o, 8, a.ndim);
  put<int32_t>(o, 12, a.B);
  for (int d = 0; d < 3; ++d) put<int64_t>(o, 16 + 8 * d, a.shape[d]);
  put<int32_t>(o, 40, a.K);
  put<int32_t>(o, 44, a.M);
  put<int32_t>(o, 48, a.chunk);
  put<int32_t>(o, 52, a.radius);
  put<int32_t>(o, 56, a.ntiers);
  put<int32_t>(o, 60, a.m);
  for (int d = 0; d < 3; ++d) put<int32_t>(o, 64 + 4 * d, a.nb[d]);
  put<int32_t>(o, 76, a.rel);
  put<double>(o, 80, sc->max_abs);
  put<double>(o, 88, a.tol);
  put<uint64_t>(o, 96, a.n_symbols);
  put<uint64_t>(o, 104, a.n_chunks);
  put<uint64_t>(o, 112, sc->n_outliers);
  put<uint64_t>(o, 120, sc->n_words);
  put<uint64_t>(o, 128, a.off_tiers);
  put<uint64_t>(o, 136, a.off_qtab);
  put<uint64_t>(o, 144, a.off_btier);
  put<uint64_t>(o, 152, a.off_chunks);
  put<uint64_t>(o, 160, a.off_codebook);
  put<uint64_t>(o, 168, sc->off_bits);
  put<uint64_t>(o, 176, sc->off_outliers);
  put<uint64_t>(o, 184, sc->total);
  put<uint32_t>(o, 192, (uint32_t)sc->codebook_bytes);
  put<uint32_t>(o, 196, (uint32_t)sc->n_runs);
  put<double>(o, 200, sc->margin);
  put<uint64_t>(o, 208, sc->off_chunk_esc);
  put<uint64_t>(o, 216, a.off_splits);
  put<uint32_t>(o, 224, (uint32_t)(a.R - 1));
  for (int i = 228; i < kHeaderBytes; ++i) o[i] = 0;
  const unsigned long long cend = sc->off_chunk_esc + (sc->n_outliers ? 4ull * a.n_chunks : 0ull);
  for (unsigned long long i = cend; i < sc->off_outliers; ++i) o[i] = 0;
  const unsigned long long oend = sc->off_outliers + 4ull * sc->n_outliers;
  for (unsigned long long i = oend; i < sc->off_bits; ++i) o[i] = 0;
  const unsigned long long wend = sc->off_bits + 4ull * sc->n_words;
  for (unsigned long long i = wend; i < sc->total; ++i) o[i] = 0;
}

__global__ void raw_header_kernel(uint8_t* o, int f64, int B, int64_t s0, int64_t s1, int64_t s2, int rel, double tol,
                                  unsigned long long total, Scalars* sc, int ndim) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kHeaderBytes; ++i) o[i] = 0;
  put<uint32_t>(o, 0, kMagic);
  put<uint16_t>(o, 4, 1);
  put<uint16_t>(o, 6, (uint16_t)(1 | (f64 ? 2 : 0)));
  put<int32_t>(o, 8, ndim);
  put<int32_t>(o, 12, B);
  put<int64_t>(o, 16, s0);
  put<int64_t>(o, 24, s1);
  put<int64_t>(o, 32, s2);
  put<int32_t>(o, 76, rel);
  const double max_abs = f64 ? __longlong_as_double((long long)sc->maxabs_bits)
                             : (double)__uint_as_float((unsigned)sc->maxabs_bits);
  put<double>(o, 80, max_abs);
  put<double>(o, 88, tol);
  put<uint64_t>(o, 168, (unsigned long long)kHeaderBytes);
  put<uint64_t>(o, 184, total);
}

// The raw fallback decided on the device: when the status says raw, the
// header of a raw stream and a copy of the field (16-byte vectors when both
// ends allow it); otherwise nothing.
template <typename T>
__global__ void __launch_bounds__(256) raw_stream_kernel(uint8_t* o, const T* __restrict__ field, int64_t nel, int f64,
                                                         int B, int64_t s0, int64_t s1, int64_t s2, int rel, double tol,
                                                         unsigned long long total, Scalars* sc, int ndim) {
  if (!(sc->status & ST_RAW)) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = 0; i < kHeaderBytes; ++i) o[i] = 0;
    put<uint32_t>(o, 0, kMagic);
    put<uint16_t>(o, 4, 1);
    put<uint16_t>(o, 6, (uint16_t)(1 | (f64 ? 2 : 0)));
    put<int32_t>(o, 8, ndim);
    put<int32_t>(o, 12, B);
    put<int64_t>(o, 16, s0);
    put<int64_t>(o, 24, s1);
    put<int64_t>(o, 32, s2);
    put<int32_t>(o, 76, rel);
    const double max_abs = f64 ? __longlong_as_double((long long)sc->maxabs_bits)
                               : (double)__uint_as_float((unsigned)sc->maxabs_bits);
    put<double>(o, 80, max_abs);
    put<double>(o, 88, tol);
    put<uint64_t>(o, 168, (unsigned long long)kHeaderBytes);
    put<uint64_t>(o, 184, total);
  }
  uint8_t* dst = o + kHeaderBytes;
  const unsigned long long bytes = (unsigned long long)nel * sizeof(T);
  const unsigned long long tid = blockIdx.x * 256ull + threadIdx.x, nth = gridDim.x * 256ull;
  const uint8_t* src = reinterpret_cast<const uint8_t*>(field);
  if (((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    const unsigned long long nv = bytes / 16;
    for (unsigned long long i = tid; i < nv; i += nth)
      reinterpret_cast<uint4*>(dst)[i] = __ldg(reinterpret_cast<const uint4*>(src) + i);
    for (unsigned long long i = nv * 16 + tid; i < bytes; i += nth) dst[i] = src[i];
  } else {
    const unsigned long long nv = bytes / sizeof(T);
    for (unsigned long long i = tid; i < nv; i += nth) reinterpret_cast<T*>(dst)[i] = field[i];
  }
}

// Decoder-side scan: chunk word counts -> word offsets; checks the total.
// One block; each warp owns a contiguous segment and walks it 32 counts at a
// time (coalesced loads, shuffle scan, running carry); the warps' totals are
// scanned across the block and a second walk writes the offsets.
__device__ __forceinline__ void word_scan_block(const unsigned* chunk_words, unsigned long long nch,
                                                unsigned long long* word_off, unsigned long long n_words, Scalars* sc) {
  __shared__ unsigned long long wt[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const unsigned long long seg = (nch + nw - 1) / nw;
  const unsigned long long a0 = min(nch, (unsigned long long)wid * seg), a1 = min(nch, a0 + seg);
  // eight loads in flight per lane (256 counts per step)
  unsigned long long tot = 0;
  for (unsigned long long b0 = a0; b0 < a1; b0 += 256) {
    unsigned v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned long long i = b0 + j * 32 + lane;
      v[j] = i < a1 ? chunk_words[i] : 0u;
    }
    unsigned long long x = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) x += v[j];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    tot += x;
  }
  if (lane == 0) wt[wid] = tot;
  __syncthreads();
  if (wid == 0) {
    unsigned long long t = lane < nw ? wt[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) wt[lane] = t;  // inclusive
  }
  __syncthreads();
  unsigned long long carry = wid ? wt[wid - 1] : 0ull;
  for (unsigned long long b0 = a0; b0 < a1; b0 += 256) {
    unsigned v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned long long i = b0 + j * 32 + lane;
      v[j] = i < a1 ? chunk_words[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const unsigned long long i = b0 + j * 32 + lane;
      unsigned long long x = v[j];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (i < a1) word_off[i] = carry + x - v[j];
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
  }
  if (threadIdx.x == 0) {
    const unsigned long long total = wt[nw - 1];
    word_off[nch] = total;
    if (total != n_words) atomicOr(&sc->status, ST_CORRUPT);
  }
}

// The decoder's three table builds in one launch, one CTA each, side by side
// on different SMs: decode tables from the codebook, word offsets of the
// chunks, and (when the stream has outliers) their per-chunk offsets.
struct TablesArgs {
  const uint8_t* runs;
  unsigned long long cb_bytes, n_runs;
  int dict;
  DecodeTables* dt;
  const unsigned* chunk_words;
  const unsigned* chunk_esc;
  unsigned long long nch, n_words, n_outliers;
  unsigned long long* word_off;
  unsigned long long* esc_off;
  Scalars* sc;
};

__global__ void __launch_bounds__(kCbThreads) tables_kernel(TablesArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (blockIdx.x == 0) decode_tables_block(a.runs, a.cb_bytes, a.n_runs, a.dict, a.dt, a.sc, smem_raw);
  else if (blockIdx.x == 1) word_scan_block(a.chunk_words, a.nch, a.word_off, a.n_words, a.sc);
  else word_scan_block(a.chunk_esc, a.nch, a.esc_off, a.n_outliers, a.sc);
}

__global__ void zero_tail_kernel(uint8_t* base, Scalars* sc) {
  // stand-alone Huffman section: zero the padding after the words
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (sc->status & ST_RAW) return;
  const unsigned long long wend = sc->off_bits + 4ull * sc->n_words;
  for (unsigned long long i = wend; i < pad8(wend); ++i) base[i] = 0;
}

namespace {

// ---------------------------------------------------------------------------
// Pipelines
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_block(int dir, int B, int K, int mode, const BlockArgs<T>& a, cudaStream_t s);
std::atomic<int> g_block_grid_cap{0};  // bm_set_block_grid_limit
template <>
cudaError_t launch_block<float>(int dir, int B, int K, int mode, const BlockArgs<float>& a, cudaStream_t s) {
  BM_LAUNCHED();
  const int cap = g_block_grid_cap.load();
  return B == 9 ? launch_block_f32_b9(dir, K, mode, a, s, num_sms(), cap)
                : launch_block_f32_b17(dir, K, mode, a, s, num_sms(), cap);
}
template <>
cudaError_t launch_block<double>(int dir, int B, int K, int mode, const BlockArgs<double>& a, cudaStream_t s) {
  BM_LAUNCHED();
  const int cap = g_block_grid_cap.load();
  return B == 9 ? launch_block_f64_b9(dir, K, mode, a, s, num_sms(), cap)
                : launch_block_f64_b17(dir, K, mode, a, s, num_sms(), cap);
}

// One restriction pass of a global level: band product and tridiagonal solve
// per line (gl_line), or the dense projection (gl_apply) for lines longer than
// gl_line takes.
template <typename T, int DIM, int FINAL, int E>
cudaError_t launch_line(const GLevel<T>& L, const ApplyShape& S, const T* in, T* out, const T* U, cudaStream_t s) {
  const GDim<T>& D = L.d[DIM];
  const size_t smem = line_smem<T>(D.n, D.c);
  static std::atomic<int> attr{0};  // largest dynamic shared memory enabled so far
  if ((int)smem > 48 * 1024 && (int)smem > attr.load()) {
    const cudaError_t e = cudaFuncSetAttribute(gl_line<T, DIM, FINAL, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    attr.store((int)smem);
  }
  const int64_t ctas = S.nb * ((S.ncol + line_tile<T>() - 1) / line_tile<T>());
  gl_line<T, DIM, FINAL, E><<<(unsigned)ctas, 256, smem, s>>>(L, S, in, out, U);
  return cudaGetLastError();
}

template <typename T, int DIM, int FINAL>
cudaError_t launch_apply(const GLevel<T>& L, const T* in, T* out, const T* U, cudaStream_t s) {
  const ApplyShape S = apply_shape(L, DIM);
  if (S.nb * S.ncol == 0) return cudaSuccess;
  switch (line_segment(L.d[DIM].c)) {
    case 1: return launch_line<T, DIM, FINAL, 1>(L, S, in, out, U, s);
    case 3: return launch_line<T, DIM, FINAL, 3>(L, S, in, out, U, s);
    case 9: return launch_line<T, DIM, FINAL, 9>(L, S, in, out, U, s);
    case 17: return launch_line<T, DIM, FINAL, 17>(L, S, in, out, U, s);
    default: break;
  }
  const int64_t ctas = S.nb * ((S.ncol + kApplyCols - 1) / kApplyCols);
  gl_apply<T, DIM, FINAL><<<(unsigned)ctas, 256, 0, s>>>(L, S, in, out, U);
  return cudaGetLastError();
}

// Outputs of the decomposition (mode 0: symbols + escapes + histogram).
template <typename T>
struct FwdOut {
  uint16_t* sym = nullptr;
  int32_t* esc = nullptr;
  T* coef = nullptr;
  unsigned* hist = nullptr;
  const uint8_t* tier = nullptr;
  const T* rq = nullptr;  // [ntiers*K + M + 1]
  int ntiers = 1;
  int radius = 0;
  Scalars* sc = nullptr;
};

// Gathered grids of the re-blocking rounds: every round but the last writes
// its own (carved from the workspace); the last writes the global levels'
// input.
template <typename T>
std::vector<T*> round_grids(const PlanHost& h, Carver& cv, T* last) {
  std::vector<T*> g;
  for (size_t r = 0; r < h.rounds.size(); ++r) {
    const RoundHost& rd = h.rounds[r];
    g.push_back(r + 1 < h.rounds.size() ? cv.take<T>((size_t)(rd.gshape[0] * rd.gshape[1] * rd.gshape[2])) : last);
  }
  return g;
}

// What run_decompose does with the fused In-cache Block stage: launch it,
// only record its arguments (and return before any launch), or skip it (the
// batched forward kernel ran it).
enum class Incache { Run, Record, Skip };

template <typename T>
bm_status run_decompose(PlanDev& P, const T* field, int mode, const FwdOut<T>& o, Carver& cv, cudaStream_t s,
                        const std::function<bm_status()>& after_block = nullptr, Incache ic = Incache::Run,
                        BlockArgs<T>* rec = nullptr) {
  const PlanHost& h = P.h;
  if (bm_status st = upload_tables<T>(P)) return st;
  const GSizes gs = gsizes(h);
  std::vector<T*> U;
  for (int l = 0; l <= h.M; ++l) U.push_back(cv.take<T>((size_t)gs.U[l]));
  T* Dbuf = cv.take<T>((size_t)gs.D);
  T* W1 = cv.take<T>((size_t)std::max<int64_t>(gs.W1, 1));
  T* W2 = cv.take<T>((size_t)std::max<int64_t>(gs.W2, 1));
  std::vector<T*> Gr = round_grids<T>(h, cv, U[0]);
  if (h.reduced) {  // a field with an extent of 1: in-cache levels on the block-major grid
    Stage st("incache_decompose");
    std::vector<T*> RB;
    for (int64_t n : gs.RB) RB.push_back(cv.take<T>((size_t)n));
    const Reblock rf = reblock_of(h, false), rc = reblock_of(h, true);
    reblock_kernel<T, 0><<<grid_for(gs.RB[0], 256), 256, 0, s>>>(rf, const_cast<T*>(field), RB[0]);
    auto& RL = rlevels<T>(P);
    for (int l = 0; l < h.K; ++l) {
      const GLevel<T>& L = RL[(size_t)l];
      const int64_t rows = (int64_t)L.d[0].n * L.d[1].n;
      const T* rq = o.rq ? o.rq + l : nullptr;
      if (mode == 0)
        gl_fwd_detail<T, 0><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, RB[l], Dbuf, o.sym, o.esc, o.coef, rq, o.radius,
                                                                       o.sc, o.tier, h.K);
      else
        gl_fwd_detail<T, 1><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, RB[l], Dbuf, o.sym, o.esc, o.coef, rq, o.radius,
                                                                       o.sc, nullptr, 0);
      BM_CUDA((launch_apply<T, 2, 0>(L, Dbuf, W1, nullptr, s)));
      BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
      gl_ident0<T, 1><<<grid_for(gs.RB[(size_t)l + 1], 256), 256, 0, s>>>(L, W2, RB[(size_t)l + 1], RB[l]);
      g_launches.fetch_add(4);
    }
    reblock_kernel<T, 1><<<grid_for(gs.RB.back(), 256), 256, 0, s>>>(rc, Gr[0], RB.back());
    g_launches.fetch_add(2);
    BM_CUDA(cudaGetLastError());
  } else if (h.generic) {  // no fused block kernel: blocked levels on each round's padded grid
    Stage st("incache_decompose");
    std::vector<T*> XP;
    for (int64_t n : gs.XP) XP.push_back(cv.take<T>((size_t)n));
    int64_t toff = 0;
    for (size_t r = 0; r < h.rounds.size(); ++r) {
      const RoundHost& rd = h.rounds[r];
      const auto& XL = xlevels<T>(P)[r];
      const XLevelHost& X0 = h.xlev[r][0];
      const T* in = r == 0 ? field : Gr[r - 1];
      const int64_t npad = X0.shape[0] * X0.shape[1] * X0.shape[2];
      pad_kernel<T, 0><<<grid_for(npad, 256), 256, 0, s>>>(in, XP[0], rd.shape[0], rd.shape[1], rd.shape[2],
                                                           X0.shape[0], X0.shape[1], X0.shape[2]);
      g_launches.fetch_add(1);
      const uint8_t* tier = o.tier ? o.tier + toff : nullptr;
      for (int l = 0; l < h.K; ++l) {
        const GLevel<T>& L = XL[(size_t)l];
        T* next = l + 1 < h.K ? XP[(size_t)l + 1] : Gr[r];
        const int64_t rows = (int64_t)L.d[0].n * L.d[1].n;
        const T* rq = o.rq ? o.rq + l : nullptr;
        if (mode == 0)
          gl_fwd_detail<T, 0><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, XP[(size_t)l], Dbuf, o.sym, o.esc,
                                                                         o.coef, rq, o.radius, o.sc, tier, h.K);
        else
          gl_fwd_detail<T, 1><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, XP[(size_t)l], Dbuf, o.sym, o.esc, o.coef,
                                                                         rq, o.radius, o.sc, nullptr, 0);
        BM_CUDA((launch_apply<T, 2, 0>(L, Dbuf, W1, nullptr, s)));
        BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
        BM_CUDA((launch_apply<T, 0, 1>(L, W2, next, XP[(size_t)l], s)));
        g_launches.fetch_add(4);
      }
      toff += rd.nblocks;
    }
    BM_CUDA(cudaGetLastError());
  } else if (ic != Incache::Skip) {
    Stage st("incache_decompose");
    int64_t toff = 0;
    for (size_t r = 0; r < h.rounds.size(); ++r) {  // each round blocks the previous round's gathered grid
      const RoundHost& rd = h.rounds[r];
      BlockArgs<T> a{};
      a.field = r == 0 ? const_cast<T*>(field) : Gr[r - 1];
      a.n0 = rd.shape[0]; a.n1 = rd.shape[1]; a.n2 = rd.shape[2];
      a.nb0 = rd.nb[0]; a.nb1 = rd.nb[1]; a.nb2 = rd.nb[2];
      a.nblocks = rd.nblocks;
      a.G = Gr[r];
      a.g1 = rd.gshape[1]; a.g2 = rd.gshape[2];
      a.sym = o.sym ? o.sym + rd.off : nullptr;
      a.esc = o.esc ? o.esc + rd.off : nullptr;
      a.coef = o.coef ? o.coef + rd.off : nullptr;
      a.tier = o.tier ? o.tier + toff : nullptr;
      a.rq = o.rq; a.hist = o.hist; a.radius = o.radius; a.sc = o.sc;
      if (ic == Incache::Record) {
        if (rec) *rec = a;
        return BM_OK;
      }
      BM_CUDA(launch_block<T>(0, h.B, h.K, mode, a, s));
      toff += rd.nblocks;
    }
  }
  if (after_block)
    if (bm_status st = after_block()) return st;
  auto& G = glevels<T>(P);
  for (int l = 0; l < h.M; ++l) {
    Stage st("global_decompose");
    const GLevel<T>& L = G[l];
    const int64_t nn = gs.U[l];
    const T* rq = o.rq ? o.rq + o.ntiers * h.K + l : nullptr;
    const int64_t rows = (int64_t)L.d[0].n * L.d[1].n;  // one warp per row, 8 rows per CTA
    if (mode == 0) gl_fwd_detail<T, 0><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, U[l], Dbuf, o.sym, o.esc, o.coef, rq, o.radius, o.sc);
    else gl_fwd_detail<T, 1><<<grid_for(rows * 32, 256, 8), 256, 0, s>>>(L, U[l], Dbuf, o.sym, o.esc, o.coef, rq, o.radius, o.sc);
    (void)nn;
    BM_LAUNCHED();
    BM_CUDA((launch_apply<T, 2, 0>(L, Dbuf, W1, nullptr, s)));
    BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
    BM_CUDA((launch_apply<T, 0, 1>(L, W2, U[l + 1], U[l], s)));
    g_launches.fetch_add(3);
  }
  {
    Stage st("coarsest");
    const int64_t cnt = gs.U[h.M];
    const T* rq = o.rq ? o.rq + o.ntiers * h.K + h.M : nullptr;
    if (mode == 0) coarsest_fwd<T, 0><<<grid_for(cnt, 256), 256, 0, s>>>(U[h.M], cnt, h.sym_off[h.M], o.sym, o.esc, o.coef, rq, o.radius, o.sc);
    else coarsest_fwd<T, 1><<<grid_for(cnt, 256), 256, 0, s>>>(U[h.M], cnt, h.sym_off[h.M], o.sym, o.esc, o.coef, rq, o.radius, o.sc);
    BM_LAUNCHED();
    BM_CUDA(cudaGetLastError());
  }
  if (mode == 0 && o.hist) {  // histogram of the global levels' and the coarsest array's symbols
    Stage st("global_histogram");
    const unsigned long long s0 = (unsigned long long)h.sym_off[0], s1 = (unsigned long long)h.n_coeffs;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms(), (int64_t)(s1 - s0) / 16384));
    BM_CUDA(launch_hist(o.sym, s0, s1, 2 * o.radius, (unsigned)o.radius, o.hist, o.sc, false, grid, s));
  }
  return BM_OK;
}

template <typename T>
struct InvIn {
  const uint16_t* sym = nullptr;
  const int32_t* esc = nullptr;
  const T* coef = nullptr;
  const uint8_t* tier = nullptr;
  const double* q = nullptr;  // [ntiers*K + M + 1]
  int ntiers = 1;
  int radius = 0;
  Scalars* sc = nullptr;      // status word for corrupt-stream checks (may be null)
};

template <typename T>
bm_status run_recompose(PlanDev& P, T* field, int mode, const InvIn<T>& in, Carver& cv, cudaStream_t s) {
  const PlanHost& h = P.h;
  if (bm_status st = upload_tables<T>(P)) return st;
  const GSizes gs = gsizes(h);
  std::vector<T*> U;
  for (int l = 0; l <= h.M; ++l) U.push_back(cv.take<T>((size_t)gs.U[l]));
  T* Dbuf = cv.take<T>((size_t)gs.D);
  T* W1 = cv.take<T>((size_t)std::max<int64_t>(gs.W1, 1));
  T* W2 = cv.take<T>((size_t)std::max<int64_t>(gs.W2, 1));
  (void)Dbuf;
  std::vector<T*> Gr = round_grids<T>(h, cv, U[0]);
  {
    Stage st("coarsest");
    const int64_t cnt = gs.U[h.M];
    const double* q = in.q ? in.q + in.ntiers * h.K + h.M : nullptr;
    if (mode == 0) coarsest_inv<T, 0><<<grid_for(cnt, 256), 256, 0, s>>>(U[h.M], cnt, h.sym_off[h.M], in.sym, in.esc, in.coef, q, in.radius);
    else coarsest_inv<T, 1><<<grid_for(cnt, 256), 256, 0, s>>>(U[h.M], cnt, h.sym_off[h.M], in.sym, in.esc, in.coef, q, in.radius);
    BM_LAUNCHED();
    BM_CUDA(cudaGetLastError());
  }
  auto& G = glevels<T>(P);
  for (int l = h.M - 1; l >= 0; --l) {
    Stage st("global_recompose");
    const GLevel<T>& L = G[l];
    const int64_t nn = gs.U[l];
    const double* q = in.q ? in.q + in.ntiers * h.K + l : nullptr;
    // U[l] <- dequantised coefficients; z = P D; coarse' = U[l+1] - z (into W1); U[l] = I coarse' + D
    if (mode == 0) gl_inv_dequant<T, 0><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius, U[l]);
    else gl_inv_dequant<T, 1><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius, U[l]);
    T* Cn = Dbuf;  // corrected coarse values (size of U[l+1] <= size of U[0])
    BM_CUDA((launch_apply<T, 2, 0>(L, U[l], W1, nullptr, s)));
    BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
    BM_CUDA((launch_apply<T, 0, 2>(L, W2, Cn, U[l + 1], s)));
    gl_inv_interp<T><<<grid_for(nn, 256), 256, 0, s>>>(L, Cn, U[l]);
    g_launches.fetch_add(5);
    BM_CUDA(cudaGetLastError());
  }
  if (h.reduced) {
    Stage st("incache_recompose");
    std::vector<T*> RB;
    for (int64_t n : gs.RB) RB.push_back(cv.take<T>((size_t)n));
    const Reblock rf = reblock_of(h, false), rc = reblock_of(h, true);
    reblock_kernel<T, 0><<<grid_for(gs.RB.back(), 256), 256, 0, s>>>(rc, Gr[0], RB.back());
    auto& RL = rlevels<T>(P);
    T* Cn = Dbuf;
    for (int l = h.K - 1; l >= 0; --l) {
      const GLevel<T>& L = RL[(size_t)l];
      const double* q = in.q ? in.q + l : nullptr;
      const int64_t nn = gs.RB[(size_t)l];
      if (mode == 0)
        gl_inv_dequant<T, 0><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius, RB[l], in.tier,
                                                                h.K, in.ntiers, in.sc);
      else
        gl_inv_dequant<T, 1><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius, RB[l]);
      BM_CUDA((launch_apply<T, 2, 0>(L, RB[l], W1, nullptr, s)));
      BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
      gl_ident0<T, 2><<<grid_for(gs.RB[(size_t)l + 1], 256), 256, 0, s>>>(L, W2, Cn, RB[(size_t)l + 1]);
      gl_inv_interp<T><<<grid_for(nn, 256), 256, 0, s>>>(L, Cn, RB[l]);
      g_launches.fetch_add(5);
    }
    reblock_kernel<T, 1><<<grid_for(gs.RB[0], 256), 256, 0, s>>>(rf, field, RB[0]);
    g_launches.fetch_add(2);
    BM_CUDA(cudaGetLastError());
  } else if (h.generic) {
    Stage st("incache_recompose");
    std::vector<T*> XP;
    for (int64_t n : gs.XP) XP.push_back(cv.take<T>((size_t)n));
    std::vector<int64_t> toff(h.rounds.size(), 0);
    for (size_t r = 1; r < h.rounds.size(); ++r) toff[r] = toff[r - 1] + h.rounds[r - 1].nblocks;
    T* Cn = Dbuf;
    for (size_t rr = h.rounds.size(); rr-- > 0;) {  // last round first: each restores its input grid
      const RoundHost& rd = h.rounds[rr];
      const auto& XL = xlevels<T>(P)[rr];
      const XLevelHost& X0 = h.xlev[rr][0];
      const uint8_t* tier = in.tier ? in.tier + toff[rr] : nullptr;
      for (int l = h.K - 1; l >= 0; --l) {
        const GLevel<T>& L = XL[(size_t)l];
        T* coarse = l + 1 < h.K ? XP[(size_t)l + 1] : Gr[rr];
        const double* q = in.q ? in.q + l : nullptr;
        const int64_t nn = (int64_t)L.d[0].n * L.d[1].n * L.d[2].n;
        if (mode == 0)
          gl_inv_dequant<T, 0><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius,
                                                                  XP[(size_t)l], tier, h.K, in.ntiers, in.sc);
        else
          gl_inv_dequant<T, 1><<<grid_for(nn, 256), 256, 0, s>>>(L, in.sym, in.esc, in.coef, q, in.radius,
                                                                  XP[(size_t)l]);
        BM_CUDA((launch_apply<T, 2, 0>(L, XP[(size_t)l], W1, nullptr, s)));
        BM_CUDA((launch_apply<T, 1, 0>(L, W1, W2, nullptr, s)));
        BM_CUDA((launch_apply<T, 0, 2>(L, W2, Cn, coarse, s)));
        gl_inv_interp<T><<<grid_for(nn, 256), 256, 0, s>>>(L, Cn, XP[(size_t)l]);
        g_launches.fetch_add(5);
      }
      T* out = rr == 0 ? field : Gr[rr - 1];
      pad_kernel<T, 1><<<grid_for(rd.shape[0] * rd.shape[1] * rd.shape[2], 256), 256, 0, s>>>(
          XP[0], out, rd.shape[0], rd.shape[1], rd.shape[2], X0.shape[0], X0.shape[1], X0.shape[2]);
      g_launches.fetch_add(1);
    }
    BM_CUDA(cudaGetLastError());
  } else {
    Stage st("incache_recompose");
    std::vector<int64_t> toff(h.rounds.size(), 0);
    for (size_t r = 1; r < h.rounds.size(); ++r) toff[r] = toff[r - 1] + h.rounds[r - 1].nblocks;
    for (size_t rr = h.rounds.size(); rr-- > 0;) {  // last round first: each restores its input grid
      const RoundHost& rd = h.rounds[rr];
      BlockArgs<T> a{};
      a.field = rr == 0 ? field : Gr[rr - 1];
      a.n0 = rd.shape[0]; a.n1 = rd.shape[1]; a.n2 = rd.shape[2];
      a.nb0 = rd.nb[0]; a.nb1 = rd.nb[1]; a.nb2 = rd.nb[2];
      a.nblocks = rd.nblocks;
      a.G = Gr[rr];
      a.g1 = rd.gshape[1]; a.g2 = rd.gshape[2];
      a.sym = in.sym ? const_cast<uint16_t*>(in.sym) + rd.off : nullptr;
      a.esc = in.esc ? const_cast<int32_t*>(in.esc) + rd.off : nullptr;
      a.coef = in.coef ? const_cast<T*>(in.coef) + rd.off : nullptr;
      a.tier = in.tier ? in.tier + toff[rr] : nullptr;
      a.q = in.q;
      a.radius = in.radius;
      a.ntiers = in.ntiers;
      a.sc = in.sc;
      BM_CUDA(launch_block<T>(1, h.B, h.K, mode, a, s));
    }
  }
  return BM_OK;
}

size_t decompose_scratch(const PlanHost& h, size_t esize) {
  const GSizes gs = gsizes(h);
  size_t b = 0;
  for (int64_t u : gs.U) b += (size_t)u * esize + 256;
  for (int64_t u : gs.RB) b += (size_t)u * esize + 256;
  for (int64_t u : gs.XP) b += (size_t)u * esize + 256;
  for (size_t r = 0; r + 1 < h.rounds.size(); ++r)
    b += (size_t)(h.rounds[r].gshape[0] * h.rounds[r].gshape[1] * h.rounds[r].gshape[2]) * esize + 256;
  b += ((size_t)gs.D + gs.W1 + gs.W2 + 3) * esize + 768;
  return b;
}

// Layout of the host-known part of a stream.
struct StreamLayout {
  unsigned long long off_tiers, off_qtab, off_btier, off_chunks, off_splits, off_codebook, nch;
  int nq;
};
StreamLayout layout(const PlanHost& h, int ntiers, int chunk) {
  StreamLayout L;
  L.nq = ntiers * h.K + h.M + 1;
  L.nch = ((unsigned long long)h.n_coeffs + chunk - 1) / chunk;
  L.off_tiers = kHeaderBytes;
  L.off_qtab = L.off_tiers + pad8(8ull * ntiers);
  L.off_btier = L.off_qtab + pad8(8ull * L.nq);
  L.off_chunks = L.off_btier + (ntiers > 1 ? pad8((unsigned long long)h.nblocks_all) : 0ull);
  L.off_splits = L.off_chunks + pad8(4ull * L.nch);
  L.off_codebook = L.off_splits + pad8(2ull * (kSplits - 1) * L.nch);
  return L;
}

// Block tiers of the rounds after the first (Sec. III-C), appended to t
// (which holds round 0's): every round-r block pushes its tier to the
// round-(r+1) blocks its gathered coarse values fall into, which keep the
// lowest (the strictest tolerance).
void propagate_tiers(const PlanHost& h, std::vector<uint8_t>& t) {
  size_t base = 0;
  for (size_t r = 0; r + 1 < h.rounds.size(); ++r) {
    const RoundHost& a = h.rounds[r];
    const RoundHost& b = h.rounds[r + 1];
    const size_t nbase = t.size();
    t.resize(nbase + (size_t)b.nblocks, 255);
    for (int64_t i0 = 0; i0 < a.nb[0]; ++i0)
      for (int64_t i1 = 0; i1 < a.nb[1]; ++i1)
        for (int64_t i2 = 0; i2 < a.nb[2]; ++i2) {
          const uint8_t v = t[base + (size_t)((i0 * a.nb[1] + i1) * a.nb[2] + i2)];
          const int64_t i[3] = {i0, i1, i2};
          int64_t lo[3], hi[3];
          for (int d = 0; d < 3; ++d) {
            lo[d] = i[d] * h.m / h.B;
            hi[d] = ((i[d] + 1) * h.m - 1) / h.B;
          }
          for (int64_t j0 = lo[0]; j0 <= hi[0]; ++j0)
            for (int64_t j1 = lo[1]; j1 <= hi[1]; ++j1)
              for (int64_t j2 = lo[2]; j2 <= hi[2]; ++j2) {
                uint8_t& w = t[nbase + (size_t)((j0 * b.nb[1] + j1) * b.nb[2] + j2)];
                w = std::min(w, v);
              }
        }
    base = nbase;
  }
}

// Pinned host staging and result of one item of a batched compress.
// Small transfers of a call (zeroed scratch, the tolerance tables from the
// pinned staging buffer, the scalars and header read back to it) done by one
// kernel through the host mapping of pinned memory rather than by copy-engine
// copies or memsets: a call then never waits behind bulk copies that the
// caller has queued on the copy engines for other data (its next field, its
// previous stream).  A span with src == nullptr is zero-filled.
struct Span {
  void* dst;
  const void* src;
  unsigned long long bytes;
};
constexpr int kMaxSpans = 8;
struct SpanArgs {
  Span r[kMaxSpans];
  int n;
};

__global__ void __launch_bounds__(256) spans_kernel(SpanArgs a) {
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x;
  for (int k = 0; k < a.n; ++k) {
    uint8_t* d = reinterpret_cast<uint8_t*>(a.r[k].dst);
    const uint8_t* src = reinterpret_cast<const uint8_t*>(a.r[k].src);
    const unsigned long long n = a.r[k].bytes;
    const uintptr_t al = reinterpret_cast<uintptr_t>(d) | (src ? reinterpret_cast<uintptr_t>(src) : 0) | (uintptr_t)n;
    if ((al & 15) == 0) {
      uint4* d4 = reinterpret_cast<uint4*>(d);
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      for (unsigned long long i = tid; i < n / 16; i += nth) d4[i] = src ? s4[i] : make_uint4(0u, 0u, 0u, 0u);
    } else if ((al & 3) == 0) {
      uint32_t* d1 = reinterpret_cast<uint32_t*>(d);
      const uint32_t* s1 = reinterpret_cast<const uint32_t*>(src);
      for (unsigned long long i = tid; i < n / 4; i += nth) d1[i] = src ? s1[i] : 0u;
    } else {
      for (unsigned long long i = tid; i < n; i += nth) d[i] = src ? src[i] : (uint8_t)0;
    }
  }
  __threadfence_system();  // stores to host memory are visible once the stream has synchronised
}

struct Spans {
  SpanArgs a{};
  void add(void* dst, const void* src, unsigned long long bytes) {
    if (bytes) a.r[a.n++] = Span{dst, src, bytes};
  }
  cudaError_t launch(cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    unsigned long long mx = 0;
    for (int k = 0; k < a.n; ++k) mx = std::max(mx, a.r[k].bytes);
    const int grid = (int)std::min<unsigned long long>((unsigned long long)num_sms() * 2, std::max(1ull, (mx + 4095) / 4096));
    spans_kernel<<<grid, 256, 0, s>>>(a);
    BM_LAUNCHED();
    return cudaGetLastError();
  }
};

// Phases of one batch item: the whole pipeline on a pool stream, or (items
// whose in-cache levels run in the batched forward kernel) a size query, the
// part before the block stage (recording the kernel's arguments) and the
// part after it.
enum BatchPhase { kWhole = 0, kQuery = 1, kPrepare = 2, kFinishA = 3, kFinishB = 4 };

struct BatchSlot {
  unsigned char* h = nullptr;  // Scalars at 0, tiers at 256, block tiers at 256 + 8*256
  unsigned char* hd = nullptr; // device-side address of h
  bool raw_now = false;        // the raw copy was chosen on the host
  unsigned long long raw_total = 0;
  int phase = kWhole;
  std::vector<double> tiers;         // kPrepare -> kFinishB: the item's tolerance tiers
  std::vector<uint8_t> btier;        // and block tiers
  bool batched = false;              // kQuery: the item can take the batched kernel
  size_t need = 0;                   // kQuery: device scratch of the item
  unsigned char* scratch = nullptr;  // kPrepare .. kFinishB: the item's own scratch
  BlockArgs<float> af{};             // kPrepare: recorded block arguments (FP32 / FP64)
  BlockArgs<double> ad{};
  QtabArgs qa{};                     // kPrepare: recorded quantiser-table arguments
  CodebookArgs cb{};                 // kFinishA: recorded codebook arguments (the batch builds them at once)
  bool cb_ready = false;
};

bm_status compress_result(const Scalars* hsc, unsigned long long raw_total, size_t* out_bytes) {
  if (hsc->status & ST_TIMEOUT) return fail(BM_ERR_CUDA, "a bounded device wait timed out (block staging or encoder look-back)");
  if (hsc->status & ST_CORRUPT) return fail(BM_ERR_CUDA, "internal error: escape count differs from the histogram");
  *out_bytes = (hsc->status & ST_RAW) ? (size_t)raw_total : (size_t)hsc->total;
  return BM_OK;
}

// Tolerance tiers of a call (Sec. III-C): the distinct values of
// min(tol, roi_b) over the blocks, ascending, and each block's tier (empty
// with a single tier), then propagated through the rounds.  Distinct values
// are collected with a cache of the last one (neighbouring blocks mostly
// share it), so a map of N blocks and t tiers costs O(N log t).
bm_status make_tiers(const PlanHost& h, double tol, const double* roi, std::vector<double>& tiers,
                     std::vector<uint8_t>& btier) {
  tiers.assign(1, tol);
  btier.clear();
  if (!roi) return BM_OK;
  tiers.clear();
  double last = -1.0;
  for (int64_t b = 0; b < h.nblocks; ++b) {
    if (!(roi[b] > 0.0) || !std::isfinite(roi[b])) return fail(BM_ERR_ARG, "ROI tolerances must be finite and > 0");
    const double v = std::min(tol, roi[b]);
    if (v == last) continue;
    last = v;
    if (std::find(tiers.begin(), tiers.end(), v) == tiers.end()) {
      if (tiers.size() == 255) return fail(BM_ERR_ARG, "more than 255 distinct tolerances");
      tiers.push_back(v);
    }
  }
  std::sort(tiers.begin(), tiers.end());
  if (tiers.size() > 1) {
    btier.resize((size_t)h.nblocks);
    double lv = -1.0;
    uint8_t lt = 0;
    for (int64_t b = 0; b < h.nblocks; ++b) {
      const double v = std::min(tol, roi[b]);
      if (v != lv) {
        lv = v;
        lt = (uint8_t)(std::lower_bound(tiers.begin(), tiers.end(), v) - tiers.begin());
      }
      btier[(size_t)b] = lt;
    }
    propagate_tiers(h, btier);
  }
  return BM_OK;
}

template <typename T>
bm_status compress_t(const T* field, const int64_t* shape, const Params& prm, double tol, int rel, const double* roi,
                     uint8_t* out, size_t cap, size_t* out_bytes, cudaStream_t s, BatchSlot* bs = nullptr) {
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  const PlanHost& h = P->h;
  if (h.n_coeffs >= (int64_t(1) << 31)) return fail(BM_ERR_UNSUPPORTED, "more than 2^31 - 1 coefficients");
  if (prm.M + prm.K > 24) return fail(BM_ERR_ARG, "too many levels");
  const bool f64 = sizeof(T) == 8;
  const int64_t nel = nel3(shape);
  const unsigned long long raw_total = kHeaderBytes + (unsigned long long)nel * sizeof(T);
  if (cap < raw_total) return fail(BM_ERR_CAPACITY, "out_capacity below bm_compress_bound()");
  // tiers: distinct min(tol, roi_i) values, ascending (one tier without a ROI
  // map); a batch item keeps them from its first phase to its last, and its
  // size query takes the largest table (255 tiers) instead
  const int phase = bs ? bs->phase : kWhole;
  std::vector<double> tiers_own;
  std::vector<uint8_t> btier_own;
  std::vector<double>& tiers = phase == kWhole ? tiers_own : bs->tiers;
  std::vector<uint8_t>& btier = phase == kWhole ? btier_own : bs->btier;
  if (phase == kWhole || phase == kPrepare)
    if (bm_status st = make_tiers(h, tol, roi, tiers, btier)) return st;
  const int ntiers = phase == kQuery ? (roi ? 255 : 1) : (int)tiers.size();
  const StreamLayout L = layout(h, ntiers, prm.chunk);
  const int dict = 2 * prm.radius;

  // scratch
  Carver cv;
  auto carve_all = [&](Carver& c, unsigned char* base) {
    c.base = base;
    c.off = 0;
  };
  Carver probe;
  carve_all(probe, nullptr);
  probe.take<Scalars>(1); probe.take<unsigned>(dict); probe.take<uint8_t>(dict); probe.take<unsigned>(dict);
  probe.take<unsigned char>(cb_big_bytes()); probe.take<unsigned>(dict);
  probe.take<double>(L.nq); probe.take<T>(L.nq); probe.take<double>(ntiers); probe.take<uint8_t>(h.nblocks_all);
  probe.take<uint16_t>((size_t)h.n_coeffs); probe.take<int32_t>((size_t)h.n_coeffs);
  probe.take<unsigned char>(256 + 16ull * L.nch);
  const size_t need = probe.off + decompose_scratch(h, sizeof(T)) + 4096;
  const size_t hneed = 256 + 8 * 256 + (size_t)h.nblocks_all + 4096;
  if (phase == kQuery) {
    bs->need = need;
    bs->batched = h.R == 1 && !h.reduced && !h.generic && fused_block(h.B) && h.K <= 4;
    return BM_OK;
  }
  Workspace* ws = nullptr;
  if (phase == kWhole) {
    if (bm_status st = get_ws(s, need, hneed, &ws)) return st;
    carve_all(cv, reinterpret_cast<unsigned char*>(ws->d));
  } else {
    carve_all(cv, bs->scratch);
    if ((phase == kFinishA || phase == kFinishB) && bs->raw_now) return BM_OK;
  }
  Scalars* sc = cv.take<Scalars>(1);
  unsigned* hist = cv.take<unsigned>(dict);
  uint8_t* lens = cv.take<uint8_t>(dict);
  unsigned* codes = cv.take<unsigned>(dict);
  unsigned char* cb_big = cv.take<unsigned char>(cb_big_bytes());
  unsigned* packed = cv.take<unsigned>(dict);
  double* qd = cv.take<double>(L.nq);
  T* rq = cv.take<T>(L.nq);
  double* dtiers = cv.take<double>(ntiers);
  uint8_t* dbt = cv.take<uint8_t>(h.nblocks_all);
  uint16_t* sym = cv.take<uint16_t>((size_t)h.n_coeffs);
  int32_t* esc = cv.take<int32_t>((size_t)h.n_coeffs);
  unsigned char* tickets = cv.take<unsigned char>(256 + 16ull * L.nch);  // ticket, then look-back status words
  unsigned long long* lb_status = reinterpret_cast<unsigned long long*>(tickets + 256);

  // pinned staging: the stream's own, or the batch item's (items of a batch
  // share streams, so each needs its own copy until the batch has synchronised)
  unsigned char* hp = bs ? bs->h : reinterpret_cast<unsigned char*>(ws->h);
  unsigned char* hpd = bs ? bs->hd : reinterpret_cast<unsigned char*>(ws->hd);  // its device-side address
  Scalars* hsc = reinterpret_cast<Scalars*>(hp);
  double* htiers = reinterpret_cast<double*>(hp + 256);
  uint8_t* hbt = hp + 256 + 8 * 256;
  std::memcpy(htiers, tiers.data(), 8 * ntiers);
  if (ntiers > 1) std::memcpy(hbt, btier.data(), btier.size());

  const bool prefix_fits = L.off_codebook <= cap;
  const bool after_block = phase == kFinishA || phase == kFinishB;
  if (!after_block) {
    Stage st("setup");
    // zeroed scalars, histogram, stream prefix and encoder tickets; the tier
    // tables read from the pinned staging buffer
    const unsigned long long nbt = (unsigned long long)h.nblocks_all;
    Spans sp;
    sp.add(sc, nullptr, sizeof(Scalars));
    sp.add(hist, nullptr, 4ull * dict);
    sp.add(dtiers, hpd + 256, 8ull * ntiers);
    if (ntiers > 1) sp.add(dbt, hpd + 256 + 8 * 256, nbt);
    if (prefix_fits) {
      if (ntiers > 1) {
        sp.add(out, nullptr, L.off_btier);
        sp.add(out + L.off_btier, hpd + 256 + 8 * 256, nbt);
        sp.add(out + L.off_btier + nbt, nullptr, L.off_codebook - L.off_btier - nbt);
      } else {
        sp.add(out, nullptr, L.off_codebook);
      }
    }
    sp.add(tickets, nullptr, 256 + 16ull * L.nch);
    BM_CUDA(sp.launch(s));
  }
  const int mgrid = (int)std::min<int64_t>((int64_t)num_sms() * BM_MAXABS_CTAS, std::max<int64_t>(1, (nel + 4095) / 4096));
  if (!after_block) {
    Stage st("maxabs");
    QtabArgs qa{};
    qa.enabled = prefix_fits;
    qa.tiers = dtiers; qa.ntiers = ntiers; qa.rel = rel; qa.K = h.K; qa.M = h.M; qa.R = h.R;
    for (size_t i = 0; i < h.A.size() && i < 24; ++i) qa.A[i] = h.A[i];
    qa.kappa = 8.0;
    qa.eps = f64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
    qa.qd = qd; qa.rq = rq; qa.f64 = f64;
    qa.out = prefix_fits ? out : nullptr;
    qa.off_tiers = L.off_tiers; qa.off_qtab = L.off_qtab; qa.sc = sc;
    if (phase == kPrepare) {
      bs->qa = qa;  // max|u| and the table are items of the batched kernel
    } else {
      maxabs_kernel<T><<<mgrid, 256, 0, s>>>(field, nel, sc, qa);
      BM_LAUNCHED();
      BM_CUDA(cudaGetLastError());
    }
  }
  if (!prefix_fits && !after_block) {  // not even the tables fit: the raw copy is the stream
    raw_header_kernel<<<1, 32, 0, s>>>(out, f64, h.B, shape[0], shape[1], shape[2], rel, tol, raw_total, sc, prm.ndim);
    BM_LAUNCHED();
    BM_CUDA(cudaMemcpyAsync(out + kHeaderBytes, field, (size_t)nel * sizeof(T), cudaMemcpyDeviceToDevice, s));
    if (bs) {
      bs->raw_now = true;
      bs->raw_total = raw_total;
      return BM_OK;
    }
    BM_CUDA(cudaStreamSynchronize(s));
    *out_bytes = (size_t)raw_total;
    return BM_OK;
  }
  FwdOut<T> fo;
  fo.sym = sym; fo.esc = esc; fo.hist = hist; fo.tier = ntiers > 1 ? dbt : nullptr; fo.rq = rq;
  fo.ntiers = ntiers; fo.radius = prm.radius; fo.sc = sc;
  // the block kernel does not count its symbols: their histogram is taken on
  // a second stream while the global levels run on the call's stream
  // (the batched kernel never counts: its items take the separate pass on
  // the item's own stream)
  auto block_hist = [&]() -> bm_status {
    if (BM_FWD_HIST && phase == kWhole) return BM_OK;
    cudaStream_t hs = s;
    const bool overlap = BM_HIST_OVERLAP && phase == kWhole;
    if (overlap) {
      if (bm_status st = ensure_aux(ws)) return st;
      BM_CUDA(cudaEventRecord(ws->ev_fork, s));
      BM_CUDA(cudaStreamWaitEvent(ws->aux, ws->ev_fork, 0));
      hs = ws->aux;
    }
    {
      Stage st("histogram", hs);
      const unsigned long long nloc = (unsigned long long)h.sym_off[0];  // the symbols of every round
      // the wide-window kernel holds most of an SM's shared memory: a share of
      // the SMs is left to the global levels running beside it
      const int hctas = dict > kHistWin ? std::max(1, num_sms() * BM_HIST_WIDE_PCT / 100) : num_sms() * BM_HIST_CTAS;
      BM_CUDA(launch_hist(sym, 0, nloc, dict, (unsigned)prm.radius, hist, sc, false, hctas, hs));
    }
    if (overlap) BM_CUDA(cudaEventRecord(ws->ev_join, ws->aux));
    return BM_OK;
  };
  if (phase == kPrepare) {  // record the block arguments; the rest follows the batched kernel
    BlockArgs<T>* rec = reinterpret_cast<BlockArgs<T>*>(f64 ? (void*)&bs->ad : (void*)&bs->af);
    return run_decompose<T>(*P, field, 0, fo, cv, s, nullptr, Incache::Record, rec);
  }
  if (phase != kFinishB) {
    const bm_status st = run_decompose<T>(*P, field, 0, fo, cv, s, block_hist,
                                          phase == kFinishA ? Incache::Skip : Incache::Run);
    // join the second stream before anything else (also on errors: no work
    // of this call may outlive it)
    if (phase == kWhole && !BM_FWD_HIST && BM_HIST_OVERLAP && ws->aux) BM_CUDA(cudaStreamWaitEvent(s, ws->ev_join, 0));
    if (st) return st;
  }
  {
    Stage st("huffman_codebook");
    CodebookArgs ca{hist, dict, lens, codes, prefix_fits ? out : nullptr, L.off_codebook, cap, sc, 1, L.nch,
                    raw_total, cb_big, packed};
    if (phase == kFinishA) {  // the batch builds every item's codebook in one launch
      bs->cb = ca;
      bs->cb_ready = true;
      return BM_OK;
    }
    if (phase != kFinishB) {
      // the table clearing, compaction and (for wide distributions) the
      // sort run on kPreCtas CTAs first; the tree itself is one CTA's work
      // (single calls only: a batch runs many codebooks side by side, and is
      // captured as a graph)
      const bool coop = BM_CB_PRESORT && bs == nullptr;
      ca.presorted = coop ? 1 : 0;
      if (coop) {
        void* kargs[] = {(void*)&ca};
        BM_CUDA(cudaLaunchCooperativeKernel((const void*)cb_presort_kernel, dim3(kPreCtas), dim3(kPreThreads), kargs,
                                            0, s));
        BM_LAUNCHED();
      }
      BM_CUDA(set_smem_once(codebook_kernel, (int)sizeof(CbSmem), g_cb_attr));
      codebook_kernel<<<1, kCbThreads, sizeof(CbSmem), s>>>(ca);
      BM_LAUNCHED();
      BM_CUDA(cudaGetLastError());
      if (coop) {  // above 8192 present symbols the codes are emitted on kPreCtas CTAs
        void* kargs[] = {(void*)&ca};
        BM_CUDA(cudaLaunchCooperativeKernel((const void*)cb_emit_kernel, dim3(kPreCtas), dim3(kPreThreads), kargs, 0,
                                            s));
        BM_LAUNCHED();
      }
    }
  }
  {
    Stage st("huffman_encode");
    FusedEncodeArgs ea{};
    ea.sym = sym; ea.esc = esc; ea.n = (unsigned long long)h.n_coeffs; ea.chunk = prm.chunk;
    ea.lens = lens; ea.codes = codes; ea.packed = packed; ea.dict = dict; ea.nch = L.nch;
    ea.ticket = reinterpret_cast<unsigned*>(tickets); ea.st = lb_status;
    ea.chunk_words = reinterpret_cast<unsigned*>(out + L.off_chunks);
    ea.splits = reinterpret_cast<uint16_t*>(out + L.off_splits);
    ea.out = out; ea.capacity = cap; ea.sc = sc;
    // the codebook picked one of four variants (the others return at once):
    // every symbol in a small window, four CTAs of eight warps per SM; every
    // symbol in the large window, or the large window with global look-ups
    // beside it, one CTA of kEncWarps warps per SM; the global table, four
    // CTAs of eight warps per SM
    constexpr int ew = kEncWarps * 32;
    const int eg = grid_for((int64_t)L.nch * 32, ew, 32 / kEncWarps);
    BM_CUDA(set_smem_once(encode_fused_kernel<kEncWarps, false, 3>, (int)enc_smem<0>(kEncWin), g_enc3_attr));
    BM_CUDA(set_smem_once(encode_fused_kernel<kEncWarps, false, 1>, (int)enc_smem<1>(kEncWin), g_enc1_attr));
    BM_CUDA(prefer_l1_once(encode_fused_kernel<8, false, 2>, g_encw_attr));
    FusedEncodeArgs e0 = ea, e1 = ea;
    e0.win = kEncWinSmall;
    e1.win = kEncWin;
    encode_fused_kernel<8, false, 0>
        <<<grid_for((int64_t)L.nch * 32, 256, 4), 256, enc_smem<0>(kEncWinSmall), s>>>(e0);
    encode_fused_kernel<kEncWarps, false, 3><<<eg, ew, enc_smem<0>(kEncWin), s>>>(e1);
    encode_fused_kernel<kEncWarps, false, 1><<<eg, ew, enc_smem<1>(kEncWin), s>>>(e1);
    encode_fused_kernel<8, false, 2><<<grid_for((int64_t)L.nch * 32, 256, 4), 256, 0, s>>>(ea);
    g_launches.fetch_add(4);
  }
  {
    Stage st("finish");
    HeaderArgs ha{};
    ha.raw_total = raw_total; ha.capacity = cap;
    ha.out = out; ha.f64 = f64; ha.B = h.B; ha.K = h.K; ha.M = h.M; ha.chunk = prm.chunk; ha.radius = prm.radius;
    ha.ntiers = ntiers; ha.m = h.m; ha.rel = rel; ha.R = h.R; ha.ndim = prm.ndim;
    for (int d = 0; d < 3; ++d) { ha.shape[d] = shape[d]; ha.nb[d] = h.nb[d]; }
    ha.tol = tol; ha.n_symbols = (unsigned long long)h.n_coeffs; ha.n_chunks = L.nch;
    ha.off_tiers = L.off_tiers; ha.off_qtab = L.off_qtab; ha.off_btier = ntiers > 1 ? L.off_btier : L.off_chunks;
    ha.off_chunks = L.off_chunks; ha.off_splits = L.off_splits; ha.off_codebook = L.off_codebook; ha.sc = sc;
    header_kernel<<<1, 32, 0, s>>>(ha);
    // a raw fallback is written on the device in the same pass (no second host round trip)
    raw_stream_kernel<T><<<mgrid, 256, 0, s>>>(out, field, nel, f64, h.B, shape[0], shape[1], shape[2], rel, tol,
                                               raw_total, sc, prm.ndim);
    g_launches.fetch_add(2);
    BM_CUDA(cudaGetLastError());
    Spans back;
    back.add(hpd, sc, sizeof(Scalars));
    BM_CUDA(back.launch(s));
  }
  if (bs) {  // the batch reads the result after its single synchronisation
    bs->raw_now = false;
    bs->raw_total = raw_total;
    return BM_OK;
  }
  BM_CUDA(cudaStreamSynchronize(s));
  return compress_result(hsc, raw_total, out_bytes);
}

// Parsed and checked header of a stream.
struct Header {
  bool raw, f64;
  int B, K, M, chunk, radius, ntiers, m, rel, R, ndim;
  int64_t shape[3];
  unsigned long long n_symbols, n_chunks, n_outliers, n_words, off_tiers, off_qtab, off_btier, off_chunks,
      off_codebook, off_bits, off_chunk_esc, off_outliers, total, off_splits;
  unsigned codebook_bytes, n_runs;
};

template <typename V>
V rd(const unsigned char* p, size_t off) {
  V v;
  std::memcpy(&v, p + off, sizeof(V));
  return v;
}

bm_status parse_header(const unsigned char* hb, size_t in_bytes, Header& H) {
  if (in_bytes < (size_t)kHeaderBytes) return fail(BM_ERR_CORRUPT, "stream shorter than its header");
  if (rd<uint32_t>(hb, 0) != kMagic) return fail(BM_ERR_CORRUPT, "bad magic");
  if (rd<uint16_t>(hb, 4) != 1) return fail(BM_ERR_CORRUPT, "unknown stream version");
  const uint16_t flags = rd<uint16_t>(hb, 6);
  H.raw = flags & 1;
  H.f64 = flags & 2;
  H.ndim = rd<int32_t>(hb, 8);
  if (H.ndim < 1 || H.ndim > 3) return fail(BM_ERR_CORRUPT, "ndim");
  H.B = rd<int32_t>(hb, 12);
  for (int d = 0; d < 3; ++d) {
    H.shape[d] = rd<int64_t>(hb, 16 + 8 * d);
    if (H.shape[d] < 1 || H.shape[d] > (int64_t(1) << 31) || (d < 3 - H.ndim && H.shape[d] != 1))
      return fail(BM_ERR_CORRUPT, "shape");
  }
  H.total = rd<uint64_t>(hb, 184);
  if (H.total != in_bytes) return fail(BM_ERR_CORRUPT, "stream length does not match its header");
  const unsigned long long nel = (unsigned long long)H.shape[0] * H.shape[1] * H.shape[2];
  if (H.raw) {
    if (in_bytes != kHeaderBytes + nel * (H.f64 ? 8 : 4)) return fail(BM_ERR_CORRUPT, "raw stream size");
    return BM_OK;
  }
  H.K = rd<int32_t>(hb, 40); H.M = rd<int32_t>(hb, 44); H.chunk = rd<int32_t>(hb, 48); H.radius = rd<int32_t>(hb, 52);
  H.ntiers = rd<int32_t>(hb, 56); H.m = rd<int32_t>(hb, 60); H.rel = rd<int32_t>(hb, 76);
  H.n_symbols = rd<uint64_t>(hb, 96); H.n_chunks = rd<uint64_t>(hb, 104); H.n_outliers = rd<uint64_t>(hb, 112);
  H.n_words = rd<uint64_t>(hb, 120);
  H.off_tiers = rd<uint64_t>(hb, 128); H.off_qtab = rd<uint64_t>(hb, 136); H.off_btier = rd<uint64_t>(hb, 144);
  H.off_chunks = rd<uint64_t>(hb, 152); H.off_codebook = rd<uint64_t>(hb, 160); H.off_bits = rd<uint64_t>(hb, 168);
  H.off_outliers = rd<uint64_t>(hb, 176);
  H.off_chunk_esc = rd<uint64_t>(hb, 208);
  H.off_splits = rd<uint64_t>(hb, 216);
  H.codebook_bytes = rd<uint32_t>(hb, 192); H.n_runs = rd<uint32_t>(hb, 196);
  H.R = (int)rd<uint32_t>(hb, 224) + 1;
  if (H.R < 1 || H.R > 8) return fail(BM_ERR_CORRUPT, "rounds");
  int kmax = 0;  // levels while a block edge still has at least 3 nodes
  for (int n = H.B; n >= 3 && n <= 64; n = n / 2 + 1) ++kmax;
  if (H.B < 3 || H.B > 64 || H.K < 1 || H.K > kmax || H.M < 0 || H.M > 16 || H.chunk < 64 ||
      H.chunk > 2048 || H.chunk % 32 || H.radius < 16 || H.radius > kMaxDict / 2 || H.ntiers < 1 || H.ntiers > 255)
    return fail(BM_ERR_CORRUPT, "header parameters out of range");
  const unsigned long long nq = (unsigned long long)H.ntiers * H.K + H.M + 1;
  if (H.off_tiers != kHeaderBytes || H.off_qtab != H.off_tiers + pad8(8ull * H.ntiers) ||
      H.off_btier != H.off_qtab + pad8(8ull * nq) || H.off_chunks < H.off_btier ||
      H.off_splits != H.off_chunks + pad8(4ull * H.n_chunks) ||
      H.off_codebook != H.off_splits + pad8(2ull * (kSplits - 1) * H.n_chunks) ||
      H.off_chunk_esc != H.off_codebook + pad8(H.codebook_bytes) ||
      H.off_outliers != H.off_chunk_esc + (H.n_outliers ? pad8(4ull * H.n_chunks) : 0ull) ||
      H.off_bits != H.off_outliers + pad8(4ull * H.n_outliers) || H.total != H.off_bits + pad8(4ull * H.n_words))
    return fail(BM_ERR_CORRUPT, "section offsets inconsistent");
  if (H.n_chunks != (H.n_symbols + H.chunk - 1) / H.chunk) return fail(BM_ERR_CORRUPT, "chunk count");
  if (H.n_outliers > H.n_symbols) return fail(BM_ERR_CORRUPT, "outlier count");
  return BM_OK;
}

bm_status read_header(const void* in, size_t in_bytes, bool is_device, cudaStream_t s, Header& H) {
  unsigned char hb[kHeaderBytes];
  if (in_bytes < (size_t)kHeaderBytes) return fail(BM_ERR_CORRUPT, "stream shorter than its header");
  if (is_device) {
    Workspace* ws = nullptr;
    if (bm_status st = get_ws(s, 1 << 12, 1 << 12, &ws)) return st;
    Spans sp;
    sp.add(ws->hd, in, kHeaderBytes);
    BM_CUDA(sp.launch(s));
    BM_CUDA(cudaStreamSynchronize(s));
    std::memcpy(hb, ws->h, kHeaderBytes);
  } else {
    std::memcpy(hb, in, kHeaderBytes);
  }
  return parse_header(hb, in_bytes, H);
}

// Decode the Huffman part of a stream into symbols + escape codes.
bm_status decode_symbols(const uint8_t* in, const Header& H, Carver& cv, uint16_t** sym_out, int32_t** esc_out,
                         Scalars** sc_out, cudaStream_t s, int stream_mode = 1) {
  Scalars* sc = cv.take<Scalars>(1);
  uint16_t* sym = cv.take<uint16_t>(H.n_symbols);
  int32_t* esc = cv.take<int32_t>(H.n_symbols);
  unsigned long long* word_off = cv.take<unsigned long long>(H.n_chunks + 1);
  unsigned long long* esc_off = cv.take<unsigned long long>(H.n_chunks + 1);
  DecodeTables* dt = cv.take<DecodeTables>(1);
  {
    Spans sp;
    sp.add(sc, nullptr, sizeof(Scalars));
    BM_CUDA(sp.launch(s));
  }
  {
    Stage st("huffman_tables");
    TablesArgs ta{};
    ta.runs = in + H.off_codebook; ta.cb_bytes = H.codebook_bytes; ta.n_runs = H.n_runs; ta.dict = 2 * H.radius;
    ta.dt = dt; ta.chunk_words = reinterpret_cast<const unsigned*>(in + H.off_chunks);
    ta.chunk_esc = reinterpret_cast<const unsigned*>(in + H.off_chunk_esc); ta.nch = H.n_chunks;
    ta.n_words = H.n_words; ta.n_outliers = H.n_outliers; ta.word_off = word_off; ta.esc_off = esc_off; ta.sc = sc;
    BM_CUDA(set_smem_once(tables_kernel, (int)sizeof(DtSmem), g_dt_attr));
    tables_kernel<<<H.n_outliers ? 3 : 2, kCbThreads, sizeof(DtSmem), s>>>(ta);
    BM_LAUNCHED();
    BM_CUDA(cudaGetLastError());
  }
  {
    Stage st("huffman_decode");
    DecodeArgs da{};
    da.words = reinterpret_cast<const unsigned*>(in + H.off_bits);
    da.n_words = H.n_words; da.word_off = word_off; da.nch = H.n_chunks; da.n = H.n_symbols; da.chunk = H.chunk;
    da.splits = reinterpret_cast<const uint16_t*>(in + H.off_splits);
    da.tab = dt; da.sym = sym; da.sc = sc;
    BM_CUDA(set_smem_once(decode_kernel, (int)kDecSmem, g_dec_attr));
    decode_kernel<<<grid_for((int64_t)H.n_chunks * kSplits, kDecThreads, dec_per_sm()), kDecThreads, kDecSmem, s>>>(da);
    BM_LAUNCHED();
    if (stream_mode && H.n_outliers) {
      escape_fixup_kernel<<<grid_for((int64_t)H.n_chunks * 32, 256, 8), 256, 0, s>>>(
          sym, H.n_symbols, H.chunk, H.n_chunks, esc_off, reinterpret_cast<const int32_t*>(in + H.off_outliers),
          H.n_outliers, esc, sc);
      BM_LAUNCHED();
    }
    BM_CUDA(cudaGetLastError());
  }
  *sym_out = sym;
  *esc_out = esc;
  *sc_out = sc;
  return BM_OK;
}

size_t decode_scratch(const Header& H) {
  return sizeof(Scalars) + 2ull * H.n_symbols + 4ull * H.n_symbols + 16ull * (H.n_chunks + 1) + sizeof(DecodeTables) +
         4096;
}

bm_status check_status(Scalars* sc, cudaStream_t s) {
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, 0, 4096, &ws)) return st;
  Spans sp;
  sp.add(ws->hd, sc, sizeof(Scalars));
  BM_CUDA(sp.launch(s));
  BM_CUDA(cudaStreamSynchronize(s));
  const Scalars* h = reinterpret_cast<const Scalars*>(ws->h);
  if (h->status & ST_CORRUPT) return fail(BM_ERR_CORRUPT, "stream failed a bound check while decoding");
  return BM_OK;
}

template <typename T>
bm_status decompress_t(const uint8_t* in, const Header& H, T* field, cudaStream_t s) {
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(H.shape, H.B, H.K, H.M, H.R, &P)) return fail(BM_ERR_CORRUPT, g_detail);
  const PlanHost& h = P->h;
  if ((unsigned long long)h.n_coeffs != H.n_symbols || h.m != H.m) return fail(BM_ERR_CORRUPT, "symbol count");
  if (H.ntiers > 1 && H.off_chunks != H.off_btier + pad8((unsigned long long)h.nblocks_all))
    return fail(BM_ERR_CORRUPT, "block tier section size");
  const size_t need = decode_scratch(H) + decompose_scratch(h, sizeof(T)) + 8192;
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, need, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  uint16_t* sym;
  int32_t* esc;
  Scalars* sc;
  if (bm_status st = decode_symbols(in, H, cv, &sym, &esc, &sc, s)) return st;
  InvIn<T> ii;
  ii.sym = sym; ii.esc = esc; ii.radius = H.radius; ii.ntiers = H.ntiers; ii.sc = sc;
  ii.q = reinterpret_cast<const double*>(in + H.off_qtab);
  ii.tier = H.ntiers > 1 ? in + H.off_btier : nullptr;
  if (bm_status st = run_recompose<T>(*P, field, 0, ii, cv, s)) return st;
  return check_status(sc, s);
}

}  // namespace
}  // namespace bm

using namespace bm;

// ===========================================================================
// C ABI
// ===========================================================================
// ---------------------------------------------------------------------------
// Transposed operators (adjoints of bm_decompose / bm_recompose)
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_block_adj(int dir, int B, int K, const BlockArgs<T>& a, cudaStream_t s);
template <>
cudaError_t launch_block_adj<float>(int dir, int B, int K, const BlockArgs<float>& a, cudaStream_t s) {
  BM_LAUNCHED();
  return launch_block_adj_f32(dir, B, K, a, s, num_sms());
}
template <>
cudaError_t launch_block_adj<double>(int dir, int B, int K, const BlockArgs<double>& a, cudaStream_t s) {
  BM_LAUNCHED();
  return launch_block_adj_f64(dir, B, K, a, s, num_sms());
}

// Expansion (M_f I M_c^-1) or restriction (I^T) along one dimension of a global level.
template <typename T>
void launch_gl_line(const GLevel<T>& L, int dim, bool expand, const T* in, T* out, cudaStream_t s) {
  const LineShape S = line_shape(L, dim);
  if (expand) {
    gl_expand<T><<<grid_for(S.nb * S.ncol, 256), 256, 0, s>>>(L.d[dim], S, in, out);
  } else {
    gl_restrict_interp<T><<<grid_for(S.nb * S.ncol * L.d[dim].c, 256), 256, 0, s>>>(L.d[dim], S, in, out);
  }
  BM_LAUNCHED();
}

// dir 0: coefficient gradients (gcoef, read) -> field gradients (gfield, written);
// dir 1: field gradients (gfield, read) -> coefficient gradients (gcoef, written).
template <typename T>
bm_status run_adjoint(PlanDev& P, int dir, T* gfield, T* gcoef, Carver& cv, cudaStream_t s) {
  const PlanHost& h = P.h;
  if (bm_status st = upload_tables<T>(P)) return st;
  const GSizes gs = gsizes(h);
  std::vector<T*> U;
  for (int l = 0; l <= h.M; ++l) U.push_back(cv.take<T>((size_t)gs.U[l]));
  T* Dbuf = cv.take<T>((size_t)gs.D);
  T* W1 = cv.take<T>((size_t)std::max<int64_t>(gs.W1, 1));
  T* W2 = cv.take<T>((size_t)std::max<int64_t>(gs.W2, 1));
  auto& G = glevels<T>(P);
  BlockArgs<T> a{};
  a.field = gfield;
  a.n0 = h.shape[0]; a.n1 = h.shape[1]; a.n2 = h.shape[2];
  a.nb0 = h.nb[0]; a.nb1 = h.nb[1]; a.nb2 = h.nb[2];
  a.nblocks = h.nblocks;
  a.G = U[0];
  a.g1 = h.gshape[1]; a.g2 = h.gshape[2];
  a.coef = gcoef;
  const int64_t ncoarsest = gs.U[h.M];
  if (dir == 0) {
    Stage st("adjoint_global");
    BM_CUDA(cudaMemcpyAsync(U[h.M], gcoef + h.sym_off[h.M], (size_t)ncoarsest * sizeof(T), cudaMemcpyDeviceToDevice, s));
    for (int l = h.M - 1; l >= 0; --l) {
      const GLevel<T>& L = G[l];
      const int64_t nn = gs.U[l], nc = gs.U[l + 1];
      // v = S_F^T g_D + P^T g_c
      gl_inv_dequant<T, 1><<<grid_for(nn, 256), 256, 0, s>>>(L, nullptr, nullptr, gcoef, nullptr, 0, U[l]);
      launch_gl_line<T>(L, 0, true, U[l + 1], W2, s);
      launch_gl_line<T>(L, 1, true, W2, W1, s);
      launch_gl_line<T>(L, 2, true, W1, Dbuf, s);
      gl_axpy<T><<<grid_for(nn, 256), 256, 0, s>>>(U[l], Dbuf, nn);
      // g_u = v + R_C^T (g_c - I^T v)
      launch_gl_line<T>(L, 2, false, U[l], W1, s);
      launch_gl_line<T>(L, 1, false, W1, W2, s);
      launch_gl_line<T>(L, 0, false, W2, Dbuf, s);
      gl_adj_correct<T><<<grid_for(nc, 256), 256, 0, s>>>(L, U[l], U[l + 1], Dbuf);
      g_launches.fetch_add(3);
      BM_CUDA(cudaGetLastError());
    }
  }
  {
    Stage st(dir == 0 ? "adjoint_incache_decompose" : "adjoint_incache_recompose");
    BM_CUDA(launch_block_adj<T>(dir, h.B, h.K, a, s));
  }
  if (dir == 1) {
    Stage st("adjoint_global");
    for (int l = 0; l < h.M; ++l) {
      const GLevel<T>& L = G[l];
      const int64_t nn = gs.U[l];
      // g_c = I^T g_u, then g_D = S_F (g_u - P^T g_c)
      launch_gl_line<T>(L, 2, false, U[l], W1, s);
      launch_gl_line<T>(L, 1, false, W1, W2, s);
      launch_gl_line<T>(L, 0, false, W2, U[l + 1], s);
      launch_gl_line<T>(L, 0, true, U[l + 1], W2, s);
      launch_gl_line<T>(L, 1, true, W2, W1, s);
      launch_gl_line<T>(L, 2, true, W1, Dbuf, s);
      gl_adj_gather<T><<<grid_for(nn, 256), 256, 0, s>>>(L, U[l], Dbuf, gcoef);
      g_launches.fetch_add(1);
      BM_CUDA(cudaGetLastError());
    }
    BM_CUDA(cudaMemcpyAsync(gcoef + h.sym_off[h.M], U[h.M], (size_t)ncoarsest * sizeof(T), cudaMemcpyDeviceToDevice, s));
  }
  return BM_OK;
}

template <typename T>
bm_status adjoint_entry(int dir, const int64_t* shape, const Params& prm, T* gfield, T* gcoef, cudaStream_t s) {
  if (prm.R != 1) return fail(BM_ERR_UNSUPPORTED, "the adjoint entry points need one round");
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  if (P->h.reduced) return fail(BM_ERR_UNSUPPORTED, "the adjoint entry points need a 3-D field without extents of 1");
  if (P->h.generic) return fail(BM_ERR_UNSUPPORTED, "the adjoint entry points need block_nodes 9 or 17");
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, decompose_scratch(P->h, sizeof(T)) + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  return run_adjoint<T>(*P, dir, gfield, gcoef, cv, s);
}

// ---------------------------------------------------------------------------
// Batched compress: the items run on a pool of streams (each with its own
// workspace), nothing synchronises until every item has been queued, and the
// results are read from per-item pinned slots afterwards.
// ---------------------------------------------------------------------------
// pool streams of a batch: the first half takes whole pipelines, the second
// half the stages after the batched forward kernel
constexpr int kBatchStreams = 16;
// A batch captured as a CUDA graph: replayed while the call's arguments (the
// key: every item's pointers, shape, dtype, tolerance, parameters and ROI
// map) and the library's scratch addresses (g_alloc_gen) stay the same.
struct BatchGraph {
  std::vector<unsigned char> key;
  cudaGraphExec_t exec = nullptr;
  std::vector<unsigned char> hstage;  // the pinned staging the graph reads (tiers, descriptors)
  std::vector<unsigned char> raw_now;
  std::vector<unsigned long long> raw_total;
  uint64_t gen = 0;
  uint64_t used = 0;
};

struct BatchCtx {
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  cudaEvent_t forks[2] = {nullptr, nullptr};  // the two halves of the pool
  unsigned char* h = nullptr;
  unsigned char* hd = nullptr;  // device-side address of h
  size_t hbytes = 0;
  unsigned char* d = nullptr;   // device scratch of the items of the batched kernel
  size_t dbytes = 0;
  cudaStream_t cap = nullptr;   // the stream a batch is captured on
  std::vector<BatchGraph> graphs;
  std::vector<std::vector<unsigned char>> seen;  // keys met once (captured when met again)
  uint64_t clock = 0;
};

// Device scratch of a batch, grown (never shrunk) under the batch lock; the
// previous batch has synchronised, so nothing uses the old buffer.
bm_status batch_scratch(BatchCtx* c, size_t bytes) {
  if (c->dbytes >= bytes) return BM_OK;
  g_alloc_gen.fetch_add(1);
  if (c->d) cudaFree(c->d);
  c->d = nullptr;
  c->dbytes = 0;
  if (cudaMalloc(&c->d, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(BM_ERR_OOM, "device scratch of the batch");
  }
  c->dbytes = bytes;
  return BM_OK;
}
std::mutex g_batch_mu;
std::map<int, BatchCtx> g_batch;

bm_status batch_ctx(size_t hbytes, BatchCtx** out) {
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  BatchCtx& c = g_batch[dev];
  if (c.streams.empty()) {
    for (int i = 0; i < kBatchStreams; ++i) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      BM_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      BM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      c.streams.push_back(st);
      c.joins.push_back(ev);
    }
    BM_CUDA(cudaEventCreateWithFlags(&c.fork, cudaEventDisableTiming));
    for (cudaEvent_t& e : c.forks) BM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  if (c.hbytes < hbytes) {
    g_alloc_gen.fetch_add(1);
    if (c.h) cudaFreeHost(c.h);
    c.h = nullptr;
    c.hd = nullptr;
    c.hbytes = 0;
    if (cudaMallocHost(&c.h, hbytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(BM_ERR_OOM, "pinned host allocation for the batch failed");
    }
    void* hd = nullptr;
    if (cudaHostGetDevicePointer(&hd, c.h, 0) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(c.h);
      c.h = nullptr;
      return fail(BM_ERR_CUDA, "pinned batch buffer is not mapped into the device address space");
    }
    c.hd = reinterpret_cast<unsigned char*>(hd);
    c.hbytes = hbytes;
  }
  *out = &c;
  return BM_OK;
}

bm_status check_item(const bm_batch_item& it, Params& prm, int64_t s3[3]) {
  if (!it.d_field || !it.d_out) return fail(BM_ERR_ARG, "NULL pointer in a batch item");
  if (bm_status st = norm_shape(it.ndim, it.shape, s3)) return st;
  if (it.dtype != BM_F32 && it.dtype != BM_F64) return fail(BM_ERR_ARG, "dtype");
  if (!(it.tol > 0.0) || !std::isfinite(it.tol)) return fail(BM_ERR_ARG, "tolerance must be finite and > 0");
  if (it.tol_mode != BM_ABS && it.tol_mode != BM_REL) return fail(BM_ERR_ARG, "tol_mode");
  if (bm_status st = check_params(&it.params, prm)) return st;
  prm.ndim = it.ndim;
  return BM_OK;
}

// ---------------------------------------------------------------------------
// Performance model and parameter selection (Sec. III-B, Eq. 1, Alg. 1)
// ---------------------------------------------------------------------------
// Seeded synthetic field for the calibration runs: a smooth part plus a
// small hashed noise (the calibration measures time, not compression).
template <typename T>
__global__ void calib_field_kernel(T* u, int64_t n0, int64_t n1, int64_t n2) {
  const int64_t n = n0 * n1 * n2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i % n2, t = i / n2, j = t % n1, l = t / n1;
    unsigned h = (unsigned)i * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    const double noise = (double)(h & 0xFFFFFF) / 16777216.0 - 0.5;
    u[i] = (T)(sin(0.13 * (double)l) * cos(0.07 * (double)j) + 0.5 * sin(0.05 * (double)k) + 0.05 * noise);
  }
}

struct CalibPoint {
  double blocks, block_ms;
  std::vector<std::pair<double, double>> global;  // (grid nodes, ms) per level
  double syms, hist_ms, ghist_syms, ghist_ms, cb_ms, enc_ms, other_ms;
};

// Eq. 1: the time of N blocks is 1/Slope + N / TP_peak (the reciprocal of
// TP(N) = N / (1/Slope + N/TP_peak), per block); a least-squares line through
// (N, time) gives both.  Other stages: straight lines in their size.
static void fit_line(const std::vector<double>& x, const std::vector<double>& y, double& a, double& b) {
  const double n = (double)x.size();
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  for (size_t i = 0; i < x.size(); ++i) {
    sx += x[i];
    sy += y[i];
    sxx += x[i] * x[i];
    sxy += x[i] * y[i];
  }
  const double den = n * sxx - sx * sx;
  b = den != 0 ? (n * sxy - sx * sy) / den : 0.0;
  a = (sy - b * sx) / n;
  if (b < 0) {  // flat: a constant
    b = 0;
    a = sy / n;
  }
  if (a < 0) a = 0;
}

// Coarse-grid shape after one level (Sec. II-B: floor(n/2)+1 nodes, none
// removed from a dimension of at most two nodes).
static int64_t coarsen(int64_t n) { return n <= 2 ? n : n / 2 + 1; }

namespace {

// One group of the batched forward kernel: items sharing dtype, B and K.
struct BatchGroup {
  bool f64;
  int B, K;
  std::vector<int> items;
};

template <typename T>
BlockArgs<T>& slot_args(BatchSlot& b) {
  return *reinterpret_cast<BlockArgs<T>*>(sizeof(T) == 8 ? (void*)&b.ad : (void*)&b.af);
}

// Descriptors of one group in pinned memory (at *hoff), copied to the device
// scratch (at *doff) and the batched kernel launched on s.
template <typename T>
bm_status launch_group(const BatchGroup& g, std::vector<BatchSlot>& slot, const std::vector<std::array<int64_t, 3>>& shp,
                       BatchCtx* ctx, size_t* hoff, size_t* doff, cudaStream_t s) {
  const size_t nf = g.items.size();
  const size_t bytes = nf * sizeof(BatchField<T>);
  BatchField<T>* hf = reinterpret_cast<BatchField<T>*>(ctx->h + *hoff);
  unsigned long long* dticket = reinterpret_cast<unsigned long long*>(ctx->d + *doff);
  BatchField<T>* df = reinterpret_cast<BatchField<T>*>(ctx->d + *doff + 256);
  unsigned long long nmax = 0, nblk = 0;
  for (size_t j = 0; j < nf; ++j) {
    BatchSlot& b = slot[(size_t)g.items[j]];
    BatchField<T>& f = hf[j];
    f.a = slot_args<T>(b);
    f.qa = b.qa;
    f.nel = nel3(shp[(size_t)g.items[j]].data());
    f.max0 = nmax;
    nmax += (unsigned long long)((f.nel + kBatchMaxChunk - 1) / kBatchMaxChunk);
  }
  for (size_t j = 0; j < nf; ++j) {
    hf[j].blk0 = nmax + nblk;
    nblk += (unsigned long long)hf[j].a.nblocks;
  }
  BatchQueue q{};
  q.ticket = dticket;
  q.n_max = nmax;
  q.n_all = nmax + nblk;
  q.nfields = (int)nf;
  BM_CUDA(cudaMemsetAsync(dticket, 0, sizeof(unsigned long long), s));
  BM_CUDA(cudaMemcpyAsync(df, hf, bytes, cudaMemcpyHostToDevice, s));
  cudaError_t e;
  if (sizeof(T) == 8)
    e = g.B == 9 ? launch_block_batch_f64_b9(g.K, reinterpret_cast<const BatchField<double>*>(df), q, s, num_sms())
                 : launch_block_batch_f64_b17(g.K, reinterpret_cast<const BatchField<double>*>(df), q, s, num_sms());
  else
    e = g.B == 9 ? launch_block_batch_f32_b9(g.K, reinterpret_cast<const BatchField<float>*>(df), q, s, num_sms())
                 : launch_block_batch_f32_b17(g.K, reinterpret_cast<const BatchField<float>*>(df), q, s, num_sms());
  BM_CUDA(e);
  BM_LAUNCHED();
  *hoff += (bytes + 255) & ~size_t(255);
  *doff += 256 + ((bytes + 255) & ~size_t(255));
  return BM_OK;
}

}  // namespace

namespace {

// Key of a batch call: the items' bytes with their ROI maps, the device and
// the block grid limit.
std::vector<unsigned char> batch_key(int n, const bm_batch_item* items, const std::vector<std::array<int64_t, 3>>& shp,
                                     const std::vector<int64_t>& nroi) {
  std::vector<unsigned char> k;
  auto put = [&](const void* p, size_t b) {
    const unsigned char* c = reinterpret_cast<const unsigned char*>(p);
    k.insert(k.end(), c, c + b);
  };
  int dev = 0;
  cudaGetDevice(&dev);
  const int cap = g_block_grid_cap.load();
  put(&dev, sizeof dev);
  put(&cap, sizeof cap);
  put(&n, sizeof n);
  for (int i = 0; i < n; ++i) {
    const bm_batch_item& it = items[i];
    put(&it.d_field, sizeof it.d_field);
    put(&it.ndim, sizeof it.ndim);
    put(shp[(size_t)i].data(), 3 * sizeof(int64_t));
    put(&it.dtype, sizeof it.dtype);
    put(&it.tol, sizeof it.tol);
    put(&it.tol_mode, sizeof it.tol_mode);
    put(&it.params, sizeof it.params);
    put(&it.d_out, sizeof it.d_out);
    put(&it.out_capacity, sizeof it.out_capacity);
    const int64_t nr = it.h_roi_tol ? nroi[(size_t)i] : -1;
    put(&nr, sizeof nr);
    if (nr > 0) put(it.h_roi_tol, (size_t)nr * sizeof(double));
  }
  return k;
}

}  // namespace

extern "C" {

const char* bm_error_string(bm_status s) {
  switch (s) {
    case BM_OK: return "ok";
    case BM_ERR_ARG: return "invalid argument";
    case BM_ERR_CUDA: return "CUDA error";
    case BM_ERR_CAPACITY: return "output capacity too small";
    case BM_ERR_CORRUPT: return "corrupt stream";
    case BM_ERR_UNSUPPORTED: return "unsupported";
    case BM_ERR_OOM: return "out of device memory";
  }
  return "unknown status";
}

const char* bm_last_error_detail(void) { return g_detail.c_str(); }

uint64_t bm_launch_count(void) { return g_launches.load(); }

void bm_set_timing(int enabled) { g_timing.store(enabled ? 1 : 0); }

void bm_set_block_grid_limit(int max_ctas) { g_block_grid_cap.store(max_ctas > 0 ? max_ctas : 0); }

int bm_stage_timeline(const char** names, float* ms, float* start_ms, int max_stages) {
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.collect();
  int n = 0;
  for (auto& r : g_timer.last) {
    if (n >= max_stages) break;
    if (names) names[n] = r.name;
    if (ms) ms[n] = r.ms;
    if (start_ms) start_ms[n] = r.start;
    ++n;
  }
  return n;
}

int bm_stage_times(const char** names, float* ms, int max_stages) {
  return bm_stage_timeline(names, ms, nullptr, max_stages);
}

size_t bm_compress_bound(int ndim, const int64_t* shape, bm_dtype dtype) {
  int64_t s3[3];
  if (norm_shape(ndim, shape, s3) != BM_OK) return 0;
  return (size_t)kHeaderBytes + (size_t)nel3(s3) * (dtype == BM_F64 ? 8 : 4);
}

bm_status bm_coeff_count(int ndim, const int64_t* shape, const bm_params* params, size_t* n_coeffs) {
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  if (n_coeffs) *n_coeffs = (size_t)P->h.n_coeffs;
  return BM_OK;
}

bm_status bm_compress(const void* d_field, int ndim, const int64_t* shape, bm_dtype dtype, double tol,
                      bm_tol_mode tol_mode, const double* h_roi_tol, const bm_params* params, void* d_out,
                      size_t out_capacity, size_t* out_bytes, void* stream) {
  if (!d_field || !d_out || !out_bytes) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  if (dtype != BM_F32 && dtype != BM_F64) return fail(BM_ERR_ARG, "dtype");
  if (!(tol > 0.0) || !std::isfinite(tol)) return fail(BM_ERR_ARG, "tolerance must be finite and > 0");
  if (tol_mode != BM_ABS && tol_mode != BM_REL) return fail(BM_ERR_ARG, "tol_mode");
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  prm.ndim = ndim;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  bm_status st;
  if (dtype == BM_F32)
    st = compress_t<float>(reinterpret_cast<const float*>(d_field), shape, prm, tol, tol_mode == BM_REL, h_roi_tol,
                           reinterpret_cast<uint8_t*>(d_out), out_capacity, out_bytes, s);
  else
    st = compress_t<double>(reinterpret_cast<const double*>(d_field), shape, prm, tol, tol_mode == BM_REL, h_roi_tol,
                            reinterpret_cast<uint8_t*>(d_out), out_capacity, out_bytes, s);
  return st;
}

bm_status bm_compress_batch(int n, const bm_batch_item* items, size_t* out_bytes, bm_status* item_status,
                            void* stream) {
  if (n < 0 || (n > 0 && (!items || !out_bytes))) return fail(BM_ERR_ARG, "NULL pointer argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  std::lock_guard<std::mutex> gb(g_batch_mu);
  g_timer.begin(s);
  std::vector<Params> prm((size_t)n);
  std::vector<size_t> slot_off((size_t)n);
  std::vector<bm_status> st((size_t)n, BM_OK);
  std::vector<std::array<int64_t, 3>> shp((size_t)n);
  std::vector<int64_t> nroi((size_t)n, 0);  // entries of each item's ROI map (first-round blocks)
  size_t hb = 0;
  for (int i = 0; i < n; ++i) {
    st[(size_t)i] = check_item(items[i], prm[(size_t)i], shp[(size_t)i].data());
    int64_t nb = 0;  // blocks of every round
    if (st[(size_t)i] == BM_OK) {
      const Params& q = prm[(size_t)i];
      int64_t m = q.B;
      for (int l = 0; l < q.K; ++l) m = m / 2 + 1;
      const int64_t* s3 = shp[(size_t)i].data();
      int64_t S[3] = {s3[0], s3[1], s3[2]};
      for (int r = 0; r < q.R; ++r) {
        int64_t nb_round = 1;
        for (int d = 0; d < 3; ++d) {
          const int64_t b = (S[d] + q.B - 1) / q.B;
          nb_round *= b;
          S[d] = b * m;
        }
        nb += nb_round;
        if (r == 0) nroi[(size_t)i] = nb_round;
      }
    }
    slot_off[(size_t)i] = hb;
    hb += (256 + 8 * 256 + (size_t)nb + 255) & ~size_t(255);
  }
  const size_t hdesc = hb;  // then the batched kernel's descriptors
  hb += (size_t)n * sizeof(BatchField<double>) + 32 * 256;
  const size_t hcb = hb;  // then the batched codebook's
  hb += (size_t)n * sizeof(CodebookArgs) + 256;
  BatchCtx* ctx = nullptr;
  if (bm_status e = batch_ctx(std::max<size_t>(hb, 256), &ctx)) return e;
  bool all_ok = true;
  for (int i = 0; i < n; ++i) all_ok = all_ok && st[(size_t)i] == BM_OK;
  const bool graphs_on = all_ok && n > 0 && !g_timing.load() && BM_BATCH_GRAPHS;
  std::vector<unsigned char> key;
  if (graphs_on) key = batch_key(n, items, shp, nroi);
  auto finish = [&](const std::vector<BatchSlot>& slot) -> bm_status {
    BM_CUDA(cudaStreamSynchronize(s));
    bm_status first = BM_OK;
    for (int i = 0; i < n; ++i) {
      out_bytes[i] = 0;
      if (st[(size_t)i] == BM_OK) {
        const BatchSlot& b = slot[(size_t)i];
        if (b.raw_now) out_bytes[i] = (size_t)b.raw_total;
        else st[(size_t)i] = compress_result(reinterpret_cast<const Scalars*>(b.h), b.raw_total, &out_bytes[i]);
      }
      if (item_status) item_status[i] = st[(size_t)i];
      if (first == BM_OK) first = st[(size_t)i];
    }
    return first;
  };
  std::vector<BatchSlot> slot((size_t)n);
  for (int i = 0; i < n; ++i) {
    slot[(size_t)i].h = ctx->h + slot_off[(size_t)i];
    slot[(size_t)i].hd = ctx->hd + slot_off[(size_t)i];
  }
  // a captured graph of this very call: restore its staging and replay it
  if (graphs_on) {
    for (BatchGraph& gph : ctx->graphs) {
      if (gph.key != key) continue;
      if (gph.gen != g_alloc_gen.load()) break;
      std::memcpy(ctx->h, gph.hstage.data(), gph.hstage.size());
      BM_CUDA(cudaGraphLaunch(gph.exec, s));
      gph.used = ++ctx->clock;
      for (int i = 0; i < n; ++i) {
        slot[(size_t)i].raw_now = gph.raw_now[(size_t)i] != 0;
        slot[(size_t)i].raw_total = gph.raw_total[(size_t)i];
      }
      return finish(slot);
    }
  }
  // the work of the call, enqueued on stream q (the call's stream, or the
  // capture stream)
  auto enqueue = [&](cudaStream_t q) -> bm_status {
    // which items take the batched forward kernel, and their scratch
    size_t dneed = 0;
    std::vector<size_t> doff((size_t)n, 0);
    std::vector<BatchGroup> groups;
    for (int i = 0; i < n; ++i) {
      if (st[(size_t)i] != BM_OK) continue;
      const bm_batch_item& it = items[i];
      BatchSlot& b = slot[(size_t)i];
      b.phase = kQuery;
      size_t dummy = 0;
      st[(size_t)i] = it.dtype == BM_F32
                          ? compress_t<float>(reinterpret_cast<const float*>(it.d_field), shp[(size_t)i].data(),
                                              prm[(size_t)i], it.tol, it.tol_mode == BM_REL, it.h_roi_tol,
                                              reinterpret_cast<uint8_t*>(it.d_out), it.out_capacity, &dummy, q, &b)
                          : compress_t<double>(reinterpret_cast<const double*>(it.d_field), shp[(size_t)i].data(),
                                               prm[(size_t)i], it.tol, it.tol_mode == BM_REL, it.h_roi_tol,
                                               reinterpret_cast<uint8_t*>(it.d_out), it.out_capacity, &dummy, q, &b);
      b.phase = kWhole;
      if (st[(size_t)i] != BM_OK || !b.batched) continue;
      doff[(size_t)i] = dneed;
      dneed += (b.need + 255) & ~size_t(255);
      const bool f64 = it.dtype == BM_F64;
      const int B = prm[(size_t)i].B, K = prm[(size_t)i].K;
      auto gi = std::find_if(groups.begin(), groups.end(),
                             [&](const BatchGroup& x) { return x.f64 == f64 && x.B == B && x.K == K; });
      if (gi == groups.end()) {
        groups.push_back(BatchGroup{f64, B, K, {}});
        gi = groups.end() - 1;
      }
      gi->items.push_back(i);
    }
    const size_t ddesc = dneed;
    if (!groups.empty()) {
      dneed += (size_t)n * sizeof(BatchField<double>) + groups.size() * 512 + 256;
      dneed += (size_t)n * sizeof(CodebookArgs) + 256;
      if (bm_status e = batch_scratch(ctx, dneed)) return e;
      for (const BatchGroup& gr : groups)
        for (int i : gr.items) {
          slot[(size_t)i].phase = kPrepare;
          slot[(size_t)i].scratch = ctx->d + doff[(size_t)i];
        }
    }
    // largest items first, so that each pool stream's workspace is sized once
    std::vector<int> order((size_t)n);
    for (int i = 0; i < n; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return nel3(shp[(size_t)a].data()) * (items[a].dtype == BM_F64 ? 2 : 1) >
             nel3(shp[(size_t)b].data()) * (items[b].dtype == BM_F64 ? 2 : 1);
    });
    constexpr int kHalf = kBatchStreams / 2;
    // items of one phase, round robin over pool streams [first, first + kHalf)
    auto run_items = [&](int want_phase, int first) {
      int k = 0;
      for (int i : order) {
        if (st[(size_t)i] != BM_OK) continue;
        BatchSlot& b = slot[(size_t)i];
        if (b.phase != want_phase) continue;
        const bm_batch_item& it = items[i];
        cudaStream_t ps = want_phase == kPrepare ? q : ctx->streams[(size_t)(first + k++ % kHalf)];
        size_t dummy = 0;
        if (it.dtype == BM_F32)
          st[(size_t)i] = compress_t<float>(reinterpret_cast<const float*>(it.d_field), shp[(size_t)i].data(),
                                            prm[(size_t)i], it.tol, it.tol_mode == BM_REL, it.h_roi_tol,
                                            reinterpret_cast<uint8_t*>(it.d_out), it.out_capacity, &dummy, ps, &b);
        else
          st[(size_t)i] = compress_t<double>(reinterpret_cast<const double*>(it.d_field), shp[(size_t)i].data(),
                                             prm[(size_t)i], it.tol, it.tol_mode == BM_REL, it.h_roi_tol,
                                             reinterpret_cast<uint8_t*>(it.d_out), it.out_capacity, &dummy, ps, &b);
      }
    };
    auto fork = [&](int first) -> bm_status {
      BM_CUDA(cudaEventRecord(ctx->forks[(size_t)(first / kHalf)], q));
      for (int j = first; j < first + kHalf; ++j)
        BM_CUDA(cudaStreamWaitEvent(ctx->streams[(size_t)j], ctx->forks[(size_t)(first / kHalf)], 0));
      return BM_OK;
    };
    // 1. the batched items' setup (one small launch each) on q
    run_items(kPrepare, 0);
    // 2. the other items' whole pipelines on the first half of the pool,
    //    beside the batched kernel
    if (bm_status e = fork(0)) return e;
    run_items(kWhole, 0);
    // 3. the batched forward kernel, one launch per (dtype, B, K), on q
    bool any = false;
    if (!groups.empty()) {
      size_t ho = hdesc, dof = ddesc;
      for (BatchGroup& gr : groups) {
        std::vector<int> live;
        for (int i : gr.items)
          if (st[(size_t)i] == BM_OK && !slot[(size_t)i].raw_now) live.push_back(i);
        for (int i : gr.items) slot[(size_t)i].phase = kFinishA;
        gr.items = live;
        if (gr.items.empty()) continue;
        any = true;
        const bm_status e = gr.f64 ? launch_group<double>(gr, slot, shp, ctx, &ho, &dof, q)
                                   : launch_group<float>(gr, slot, shp, ctx, &ho, &dof, q);
        if (e) return e;
      }
    }
    // 4. the batched items' histograms and global levels on the second half,
    //    their codebooks in one launch (one CTA each) on q, then their
    //    encoders and headers on the second half again
    if (any || !groups.empty()) {
      if (bm_status e = fork(kHalf)) return e;
      run_items(kFinishA, kHalf);
      for (int j = kHalf; j < kBatchStreams; ++j) {
        BM_CUDA(cudaEventRecord(ctx->joins[(size_t)j], ctx->streams[(size_t)j]));
        BM_CUDA(cudaStreamWaitEvent(q, ctx->joins[(size_t)j], 0));
      }
      CodebookArgs* hc = reinterpret_cast<CodebookArgs*>(ctx->h + hcb);
      int ncb = 0;
      for (int i : order)
        if (st[(size_t)i] == BM_OK && slot[(size_t)i].phase == kFinishA && slot[(size_t)i].cb_ready)
          hc[ncb++] = slot[(size_t)i].cb;
      if (ncb) {
        const size_t dcb = ddesc + (size_t)n * sizeof(BatchField<double>) + groups.size() * 512 + 256;
        CodebookArgs* dc = reinterpret_cast<CodebookArgs*>(ctx->d + dcb);
        BM_CUDA(cudaMemcpyAsync(dc, hc, (size_t)ncb * sizeof(CodebookArgs), cudaMemcpyHostToDevice, q));
        BM_CUDA(set_smem_once(codebook_batch_kernel, (int)sizeof(CbSmem), g_cbb_attr));
        codebook_batch_kernel<<<(unsigned)ncb, kCbThreads, sizeof(CbSmem), q>>>(dc);
        BM_LAUNCHED();
        BM_CUDA(cudaGetLastError());
      }
      for (int i : order)
        if (slot[(size_t)i].phase == kFinishA) slot[(size_t)i].phase = kFinishB;
      if (bm_status e = fork(kHalf)) return e;
      run_items(kFinishB, kHalf);
    }
    // 5. every pool stream back into q
    for (size_t j = 0; j < ctx->streams.size(); ++j) {
      BM_CUDA(cudaEventRecord(ctx->joins[j], ctx->streams[j]));
      BM_CUDA(cudaStreamWaitEvent(q, ctx->joins[j], 0));
    }
    return BM_OK;
  };
  // capture the call when its key was met before (scratch is sized by then)
  bool capture = false;
  if (graphs_on) {
    auto it = std::find(ctx->seen.begin(), ctx->seen.end(), key);
    if (it != ctx->seen.end()) {
      capture = true;
      ctx->seen.erase(it);
    } else {
      ctx->seen.push_back(key);
      if (ctx->seen.size() > 8) ctx->seen.erase(ctx->seen.begin());
    }
  }
  if (capture) {
    if (!ctx->cap) BM_CUDA(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    const uint64_t gen0 = g_alloc_gen.load();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    bm_status e = BM_OK;
    if (ok) {
      e = enqueue(ctx->cap);
      ok = cudaStreamEndCapture(ctx->cap, &graph) == cudaSuccess && e == BM_OK && graph;
      ok = ok && g_alloc_gen.load() == gen0;
      for (int i = 0; i < n && ok; ++i) ok = st[(size_t)i] == BM_OK;
      ok = ok && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    }
    if (graph) cudaGraphDestroy(graph);
    if (ok) {
      BatchGraph gph;
      gph.key = std::move(key);
      gph.exec = exec;
      gph.hstage.assign(ctx->h, ctx->h + hb);
      gph.gen = gen0;
      gph.used = ++ctx->clock;
      for (int i = 0; i < n; ++i) {
        gph.raw_now.push_back(slot[(size_t)i].raw_now ? 1 : 0);
        gph.raw_total.push_back(slot[(size_t)i].raw_total);
      }
      if (ctx->graphs.size() >= 4) {  // least recently used out
        auto lru = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](const BatchGraph& a, const BatchGraph& b) { return a.used < b.used; });
        cudaGraphExecDestroy(lru->exec);
        ctx->graphs.erase(lru);
      }
      ctx->graphs.push_back(std::move(gph));
      BM_CUDA(cudaGraphLaunch(exec, s));
      return finish(slot);
    }
    // the capture failed: clear its errors and run the call directly
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();
    for (int i = 0; i < n; ++i) {
      st[(size_t)i] = BM_OK;
      BatchSlot fresh;
      fresh.h = slot[(size_t)i].h;
      fresh.hd = slot[(size_t)i].hd;
      slot[(size_t)i] = fresh;
    }
  }
  // graphs holding stale scratch addresses are of no further use
  for (size_t j = 0; j < ctx->graphs.size();) {
    if (ctx->graphs[j].gen != g_alloc_gen.load()) {
      cudaGraphExecDestroy(ctx->graphs[j].exec);
      ctx->graphs.erase(ctx->graphs.begin() + (long)j);
    } else {
      ++j;
    }
  }
  if (bm_status e = enqueue(s)) {
    cudaStreamSynchronize(s);
    return e;
  }
  return finish(slot);
}

bm_status bm_perf_model_fit(bm_dtype dtype, int block_nodes, bm_perf_model* model, void* stream) {
  if (!model) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (dtype != BM_F32 && dtype != BM_F64) return fail(BM_ERR_ARG, "dtype");
  bm_params bp{};
  bp.block_nodes = block_nodes;
  Params prm;
  if (bm_status st = check_params(&bp, prm)) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t esize = dtype == BM_F64 ? 8 : 4;
  // fields of 1^3 .. 22^3 blocks (up to ~0.8 GB of FP32 input at B = 17)
  const int nb_list[] = {1, 2, 3, 4, 6, 8, 10, 12, 14, 16, 19, 22};
  const int64_t emax = (int64_t)22 * prm.B;
  const size_t fbytes = (size_t)(emax * emax * emax) * esize;
  const size_t obytes = kHeaderBytes + fbytes;
  void* dfield = nullptr;
  void* dout = nullptr;
  BM_CUDA(cudaMalloc(&dfield, fbytes));
  if (cudaMalloc(&dout, obytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dfield);
    return fail(BM_ERR_OOM, "calibration buffers");
  }
  std::vector<CalibPoint> pts;
  bm_status st = BM_OK;
  const int prev_timing = g_timing.load();
  g_timing.store(1);
  for (int nb : nb_list) {
    const int64_t e = (int64_t)nb * prm.B;
    const int64_t shape[3] = {e, e, e};
    if (dtype == BM_F64) calib_field_kernel<double><<<grid_for(e * e * e, 256), 256, 0, s>>>((double*)dfield, e, e, e);
    else calib_field_kernel<float><<<grid_for(e * e * e, 256), 256, 0, s>>>((float*)dfield, e, e, e);
    CalibPoint cp{};
    for (int rep = 0; rep < 3 && st == BM_OK; ++rep) {  // warm-up, then two timed calls (the second kept)
      size_t nbytes = 0;
      {
        std::lock_guard<std::mutex> g(g_timer_mu);
        g_timer.begin(s);
        st = dtype == BM_F64 ? compress_t<double>((const double*)dfield, shape, prm, 1e-3, 1, nullptr,
                                                   (uint8_t*)dout, obytes, &nbytes, s)
                             : compress_t<float>((const float*)dfield, shape, prm, 1e-3, 1, nullptr,
                                                 (uint8_t*)dout, obytes, &nbytes, s);
        g_timer.collect();
      }
      if (st != BM_OK || rep == 0) continue;
      PlanDev* P = nullptr;
      if ((st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) != BM_OK) break;
      const GSizes gs = gsizes(P->h);
      cp = CalibPoint{};
      cp.blocks = (double)P->h.nblocks;
      cp.syms = (double)P->h.nblocks * (double)P->h.per_block;
      cp.ghist_syms = (double)(P->h.n_coeffs - P->h.sym_off[0]);
      int gl = 0;
      for (auto& r : g_timer.last) {
        const std::string name = r.name;
        if (name == "incache_decompose") cp.block_ms = r.ms;
        else if (name == "global_decompose") cp.global.push_back({(double)gs.U[(size_t)gl++], (double)r.ms});
        else if (name == "histogram") cp.hist_ms = r.ms;
        else if (name == "global_histogram") cp.ghist_ms = r.ms;
        else if (name == "huffman_codebook") cp.cb_ms = r.ms;
        else if (name == "huffman_encode") cp.enc_ms = r.ms;
        else cp.other_ms += r.ms;
      }
    }
    if (st != BM_OK) break;
    pts.push_back(cp);
  }
  g_timing.store(prev_timing);
  cudaFree(dfield);
  cudaFree(dout);
  if (st != BM_OK) return st;
  std::vector<double> x, y;
  for (auto& p : pts) { x.push_back(p.blocks); y.push_back(p.block_ms); }
  double a = 0, b = 0;
  fit_line(x, y, a, b);
  model->block_latency_ms = a;                  // 1 / Slope
  model->block_peak_per_ms = b > 0 ? 1.0 / b : 0.0;  // TP_peak (blocks per ms)
  x.clear(); y.clear();
  for (auto& p : pts) for (auto& g : p.global) { x.push_back(g.first); y.push_back(g.second); }
  fit_line(x, y, model->global_ms, model->global_ms_per_node);
  x.clear(); y.clear();
  for (auto& p : pts) { x.push_back(p.syms); y.push_back(p.hist_ms); x.push_back(p.ghist_syms); y.push_back(p.ghist_ms); }
  fit_line(x, y, model->hist_ms, model->hist_ms_per_symbol);
  x.clear(); y.clear();
  for (auto& p : pts) { x.push_back(p.syms + p.ghist_syms); y.push_back(p.enc_ms); }
  fit_line(x, y, model->encode_ms, model->encode_ms_per_symbol);
  double cb = 0, other = 0;
  for (auto& p : pts) { cb += p.cb_ms; other += p.other_ms; }
  model->codebook_ms = cb / (double)pts.size();
  model->other_ms = other / (double)pts.size();
  model->block_nodes = prm.B;
  model->incache_levels = prm.K;
  model->dtype = dtype;
  return BM_OK;
}

double bm_perf_model_knee(const bm_perf_model* m, double fraction) {
  // TP(N) / TP_peak = N / (N + N0), N0 = TP_peak / Slope: the fraction is
  // reached at N = N0 * fraction / (1 - fraction)
  if (!m || !(fraction > 0.0) || !(fraction < 1.0)) return 0.0;
  const double n0 = m->block_peak_per_ms * m->block_latency_ms;
  return n0 * fraction / (1.0 - fraction);
}

bm_status bm_predict_ms(const bm_perf_model* m, int ndim, const int64_t* shape, const bm_params* params,
                        double* ms) {
  if (!m || !ms) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  const PlanHost& h = P->h;
  const GSizes gs = gsizes(h);
  // the in-cache levels (quantisation fused) follow Eq. 1; a model fitted
  // for K levels is scaled by the share of a block's work the other K keep
  // (each level's work is ~ its node count)
  double kscale = 1.0;
  if (m->incache_levels > 0 && m->incache_levels != prm.K) {
    auto work = [&](int K) {
      double w = 0, n = prm.B;
      for (int l = 0; l < K; ++l) { w += n * n * n; n = (double)coarsen((int64_t)n); }
      return w;
    };
    kscale = work(prm.K) / work(m->incache_levels);
  }
  const double nb = (double)h.nblocks;
  double t = kscale * (m->block_latency_ms + (m->block_peak_per_ms > 0 ? nb / m->block_peak_per_ms : 0.0));
  for (int l = 0; l < h.M; ++l) t += m->global_ms + m->global_ms_per_node * (double)gs.U[(size_t)l];
  const double syms = (double)h.n_coeffs;
  t += std::max(m->hist_ms, m->hist_ms_per_symbol * syms);
  t += m->codebook_ms;
  t += std::max(m->encode_ms, m->encode_ms_per_symbol * syms);
  t += m->other_ms;
  *ms = t;
  return BM_OK;
}

bm_status bm_select_params(const bm_perf_model* m, int ndim, const int64_t* shape, double budget_ms,
                           bm_params* out, double* predicted_ms) {
  if (!m || !out) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  const int B = m->block_nodes ? m->block_nodes : 17;
  const int kmax = B == 9 ? 3 : 4;
  bool found = false;
  int bestK = 0, bestM = -1;
  double bestT = 0;
  for (int K = 1; K <= kmax; ++K) {
    // block-coarse grid after K levels, then the global levels that still coarsen
    int64_t mb = B;
    for (int l = 0; l < K; ++l) mb = coarsen(mb);
    int64_t g[3];
    for (int d = 0; d < 3; ++d) g[d] = ((shape[d] + B - 1) / B) * mb;
    int mmax = 0;
    while (mmax < 16 && (g[0] > 2 || g[1] > 2 || g[2] > 2)) {
      for (int d = 0; d < 3; ++d) g[d] = coarsen(g[d]);
      ++mmax;
    }
    for (int M = 0; M <= mmax; ++M) {
      bm_params p{};
      p.block_nodes = B;
      p.incache_levels = K;
      p.global_levels = M ? M : -1;
      double t = 0;
      if (bm_predict_ms(m, ndim, shape, &p, &t) != BM_OK) continue;
      if (t > budget_ms) continue;
      // Alg. 1: the feasible pair that is largest in (M, -K)
      if (!found || M > bestM || (M == bestM && K < bestK)) {
        found = true;
        bestK = K;
        bestM = M;
        bestT = t;
      }
    }
  }
  if (!found) return fail(BM_ERR_UNSUPPORTED, "no (levels, global levels) pair meets the time budget");
  *out = bm_params{};
  out->block_nodes = B;
  out->incache_levels = bestK;
  out->global_levels = bestM ? bestM : -1;
  if (predicted_ms) *predicted_ms = bestT;
  return BM_OK;
}

bm_status bm_stream_info(const void* in, size_t in_bytes, int in_is_device, int* ndim, int64_t shape[3],
                         bm_dtype* dtype, size_t* n_coeffs) {
  if (!in) return fail(BM_ERR_ARG, "NULL stream");
  Header H{};
  if (bm_status st = read_header(in, in_bytes, in_is_device != 0, nullptr, H)) return st;
  if (ndim) *ndim = H.ndim;
  if (shape) {  // the field's own extents first; unused entries 0
    for (int d = 0; d < 3; ++d) shape[d] = 0;
    for (int d = 0; d < H.ndim; ++d) shape[d] = H.shape[3 - H.ndim + d];
  }
  if (dtype) *dtype = H.f64 ? BM_F64 : BM_F32;
  if (n_coeffs) *n_coeffs = H.raw ? 0 : (size_t)H.n_symbols;
  return BM_OK;
}

bm_status bm_decompress(const void* d_in, size_t in_bytes, void* d_field, void* stream) {
  if (!d_in || !d_field) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (reinterpret_cast<uintptr_t>(d_in) % 8) return fail(BM_ERR_ARG, "stream pointer must be 8-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  Header H{};
  if (bm_status st = read_header(d_in, in_bytes, true, s, H)) return st;
  const uint8_t* in = reinterpret_cast<const uint8_t*>(d_in);
  if (H.raw) {
    const size_t nb = (size_t)nel3(H.shape) * (H.f64 ? 8 : 4);
    BM_CUDA(cudaMemcpyAsync(d_field, in + kHeaderBytes, nb, cudaMemcpyDeviceToDevice, s));
    BM_CUDA(cudaStreamSynchronize(s));
    return BM_OK;
  }
  return H.f64 ? decompress_t<double>(in, H, reinterpret_cast<double*>(d_field), s)
               : decompress_t<float>(in, H, reinterpret_cast<float*>(d_field), s);
}

bm_status bm_decompose(const void* d_field, int ndim, const int64_t* shape, bm_dtype dtype, const bm_params* params,
                       void* d_coeffs, void* stream) {
  if (!d_field || !d_coeffs) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  const size_t esize = dtype == BM_F64 ? 8 : 4;
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, decompose_scratch(P->h, esize) + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  if (dtype == BM_F64) {
    FwdOut<double> o;
    o.coef = reinterpret_cast<double*>(d_coeffs);
    return run_decompose<double>(*P, reinterpret_cast<const double*>(d_field), 1, o, cv, s);
  }
  FwdOut<float> o;
  o.coef = reinterpret_cast<float*>(d_coeffs);
  return run_decompose<float>(*P, reinterpret_cast<const float*>(d_field), 1, o, cv, s);
}

bm_status bm_recompose(const void* d_coeffs, int ndim, const int64_t* shape, bm_dtype dtype, const bm_params* params,
                       void* d_field, void* stream) {
  if (!d_field || !d_coeffs) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  PlanDev* P = nullptr;
  if (bm_status st = get_plan(shape, prm.B, prm.K, prm.M, prm.R, &P)) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  const size_t esize = dtype == BM_F64 ? 8 : 4;
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, decompose_scratch(P->h, esize) + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  if (dtype == BM_F64) {
    InvIn<double> in;
    in.coef = reinterpret_cast<const double*>(d_coeffs);
    return run_recompose<double>(*P, reinterpret_cast<double*>(d_field), 1, in, cv, s);
  }
  InvIn<float> in;
  in.coef = reinterpret_cast<const float*>(d_coeffs);
  return run_recompose<float>(*P, reinterpret_cast<float*>(d_field), 1, in, cv, s);
}

bm_status bm_decompose_adjoint(const void* d_coeff_grad, int ndim, const int64_t* shape, bm_dtype dtype,
                               const bm_params* params, void* d_field_grad, void* stream) {
  if (!d_coeff_grad || !d_field_grad) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == BM_F64)
    return adjoint_entry<double>(0, shape, prm, reinterpret_cast<double*>(d_field_grad),
                                 const_cast<double*>(reinterpret_cast<const double*>(d_coeff_grad)), s);
  return adjoint_entry<float>(0, shape, prm, reinterpret_cast<float*>(d_field_grad),
                              const_cast<float*>(reinterpret_cast<const float*>(d_coeff_grad)), s);
}

bm_status bm_recompose_adjoint(const void* d_field_grad, int ndim, const int64_t* shape, bm_dtype dtype,
                               const bm_params* params, void* d_coeff_grad, void* stream) {
  if (!d_coeff_grad || !d_field_grad) return fail(BM_ERR_ARG, "NULL pointer argument");
  int64_t s3_[3];
  if (bm_status st = norm_shape(ndim, shape, s3_)) return st;
  shape = s3_;
  Params prm;
  if (bm_status st = check_params(params, prm)) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == BM_F64)
    return adjoint_entry<double>(1, shape, prm, const_cast<double*>(reinterpret_cast<const double*>(d_field_grad)),
                                 reinterpret_cast<double*>(d_coeff_grad), s);
  return adjoint_entry<float>(1, shape, prm, const_cast<float*>(reinterpret_cast<const float*>(d_field_grad)),
                              reinterpret_cast<float*>(d_coeff_grad), s);
}

bm_status bm_stream_codes(const void* d_in, size_t in_bytes, int32_t* d_codes, void* stream) {
  if (!d_in || !d_codes) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (reinterpret_cast<uintptr_t>(d_in) % 8) return fail(BM_ERR_ARG, "stream pointer must be 8-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  Header H{};
  if (bm_status st = read_header(d_in, in_bytes, true, s, H)) return st;
  if (H.raw) return fail(BM_ERR_ARG, "raw stream has no codes");
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, decode_scratch(H) + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  uint16_t* sym;
  int32_t* esc;
  Scalars* sc;
  const uint8_t* in = reinterpret_cast<const uint8_t*>(d_in);
  if (bm_status st = decode_symbols(in, H, cv, &sym, &esc, &sc, s)) return st;
  codes_from_symbols_kernel<<<grid_for((int64_t)H.n_symbols, 256), 256, 0, s>>>(sym, esc, H.n_symbols, H.radius, d_codes);
  BM_LAUNCHED();
  BM_CUDA(cudaGetLastError());
  return check_status(sc, s);
}

bm_status bm_huffman_encode(const uint16_t* d_symbols, uint64_t n, int dict_size, int chunk_symbols, void* d_out,
                            size_t out_capacity, uint64_t sizes_out[5], void* stream) {
  if (!d_symbols || !d_out || !sizes_out) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (n == 0 || n >= (uint64_t(1) << 31)) return fail(BM_ERR_ARG, "symbol count must be in [1, 2^31)");
  if (dict_size < 2 || dict_size > kMaxDict) return fail(BM_ERR_ARG, "dict_size must be in [2, 65536]");
  if (chunk_symbols < 64 || chunk_symbols > 2048 || chunk_symbols % 32) return fail(BM_ERR_ARG, "chunk_symbols");
  if (reinterpret_cast<uintptr_t>(d_out) % 8) return fail(BM_ERR_ARG, "output pointer must be 8-byte aligned");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  const unsigned long long nch = (n + chunk_symbols - 1) / chunk_symbols;
  const unsigned long long off_sp = pad8(4ull * nch);
  const unsigned long long off_cb = off_sp + pad8(2ull * (kSplits - 1) * nch);
  if (off_cb > out_capacity) return fail(BM_ERR_CAPACITY, "capacity below the chunk table");
  Carver probe;
  probe.take<Scalars>(1); probe.take<unsigned>(dict_size); probe.take<uint8_t>(dict_size);
  probe.take<unsigned>(dict_size); probe.take<unsigned>(nch); probe.take<unsigned char>(256 + 16ull * nch);
  probe.take<unsigned char>(cb_big_bytes()); probe.take<unsigned>(dict_size);
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, probe.off + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  Scalars* sc = cv.take<Scalars>(1);
  unsigned* hist = cv.take<unsigned>(dict_size);
  uint8_t* lens = cv.take<uint8_t>(dict_size);
  unsigned* codes = cv.take<unsigned>(dict_size);
  unsigned char* tickets = cv.take<unsigned char>(256 + 16ull * nch);
  unsigned char* cb_big = cv.take<unsigned char>(cb_big_bytes());
  unsigned* packed = cv.take<unsigned>(dict_size);
  uint8_t* out = reinterpret_cast<uint8_t*>(d_out);
  BM_CUDA(cudaMemsetAsync(sc, 0, sizeof(Scalars), s));
  BM_CUDA(cudaMemsetAsync(hist, 0, 4ull * dict_size, s));
  BM_CUDA(cudaMemsetAsync(out, 0, off_cb, s));
  BM_CUDA(cudaMemsetAsync(tickets, 0, 256 + 16ull * nch, s));
  {
    Stage st("huffman_histogram");
    BM_CUDA(launch_hist(d_symbols, 0, n, dict_size, (unsigned)(dict_size / 2), hist, sc, true,
                        grid_for((int64_t)n, 256, 4), s));
  }
  {
    Stage st("huffman_codebook");
    CodebookArgs ca{hist, dict_size, lens, codes, out, off_cb, out_capacity, sc, 0, nch, ~0ull, cb_big, packed};
    BM_CUDA(set_smem_once(codebook_kernel, (int)sizeof(CbSmem), g_cb_attr));
    codebook_kernel<<<1, kCbThreads, sizeof(CbSmem), s>>>(ca);
    BM_LAUNCHED();
  }
  {
    Stage st("huffman_encode");
    FusedEncodeArgs ea{};
    ea.sym = d_symbols; ea.esc = nullptr; ea.n = n; ea.chunk = chunk_symbols; ea.lens = lens; ea.codes = codes;
    ea.dict = dict_size; ea.nch = nch; ea.ticket = reinterpret_cast<unsigned*>(tickets);
    ea.st = reinterpret_cast<unsigned long long*>(tickets + 256);
    ea.chunk_words = reinterpret_cast<unsigned*>(out); ea.out = out;
    ea.splits = reinterpret_cast<uint16_t*>(out + off_sp);
    ea.capacity = out_capacity; ea.sc = sc;
    ea.packed = packed;
    ea.win = kEncWinSmall;
    if (dict_size <= kEncWinSmall) {
      encode_fused_kernel<8, true, 0>
          <<<grid_for((int64_t)nch * 32, 256, 4), 256, enc_smem<0>(kEncWinSmall), s>>>(ea);
    } else {
      BM_CUDA(prefer_l1_once(encode_fused_kernel<8, true, 2>, g_encc_attr));
      encode_fused_kernel<8, true, 2><<<grid_for((int64_t)nch * 32, 256, 4), 256, 0, s>>>(ea);
    }
    encode_finish_kernel<<<1, 32, 0, s>>>(~0ull, out_capacity, sc);
    zero_tail_kernel<<<1, 32, 0, s>>>(out, sc);
    g_launches.fetch_add(3);
    BM_CUDA(cudaGetLastError());
  }
  Scalars* hsc = reinterpret_cast<Scalars*>(ws->h);
  BM_CUDA(cudaMemcpyAsync(hsc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  BM_CUDA(cudaStreamSynchronize(s));
  if (hsc->status & ST_TIMEOUT) return fail(BM_ERR_CUDA, "encoder look-back wait timed out");
  if (hsc->status & ST_CORRUPT) return fail(BM_ERR_ARG, "a symbol is not below dict_size");
  if (hsc->status & (ST_RAW | ST_CAPACITY)) return fail(BM_ERR_CAPACITY, "output capacity too small");
  sizes_out[0] = hsc->codebook_bytes;
  sizes_out[1] = hsc->n_runs;
  sizes_out[2] = nch;
  sizes_out[3] = hsc->n_words;
  sizes_out[4] = pad8(hsc->off_bits + 4ull * hsc->n_words);
  return BM_OK;
}

bm_status bm_huffman_decode(const void* d_section, const uint64_t sizes[5], uint64_t n, int dict_size,
                            int chunk_symbols, uint16_t* d_symbols, void* stream) {
  if (!d_section || !sizes || !d_symbols) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (dict_size < 2 || dict_size > kMaxDict) return fail(BM_ERR_ARG, "dict_size must be in [2, 65536]");
  if (chunk_symbols < 64 || chunk_symbols > 2048 || chunk_symbols % 32) return fail(BM_ERR_ARG, "chunk_symbols");
  if (reinterpret_cast<uintptr_t>(d_section) % 8) return fail(BM_ERR_ARG, "section pointer must be 8-byte aligned");
  const unsigned long long nch = (n + chunk_symbols - 1) / chunk_symbols;
  if (sizes[2] != nch) return fail(BM_ERR_CORRUPT, "chunk count does not match n");
  const unsigned long long off_sp = pad8(4ull * nch);
  const unsigned long long off_cb = off_sp + pad8(2ull * (kSplits - 1) * nch), off_w = off_cb + pad8(sizes[0]);
  if (sizes[4] < off_w + 4ull * sizes[3]) return fail(BM_ERR_CORRUPT, "section sizes inconsistent");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> g(g_timer_mu);
  g_timer.begin(s);
  Header H{};
  H.n_symbols = n; H.n_chunks = nch; H.n_words = sizes[3]; H.n_outliers = 0; H.off_chunks = 0; H.off_splits = off_sp;
  H.off_codebook = off_cb; H.off_bits = off_w; H.codebook_bytes = (unsigned)sizes[0]; H.n_runs = (unsigned)sizes[1];
  H.radius = dict_size / 2;  // only 2*radius = dict is used by the decoder
  H.chunk = chunk_symbols;
  Workspace* ws = nullptr;
  if (bm_status st = get_ws(s, decode_scratch(H) + 4096, 4096, &ws)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(ws->d);
  uint16_t* sym;
  int32_t* esc;
  Scalars* sc;
  if (dict_size & 1) return fail(BM_ERR_ARG, "dict_size must be even");
  if (bm_status st = decode_symbols(reinterpret_cast<const uint8_t*>(d_section), H, cv, &sym, &esc, &sc, s, 0))
    return st;
  BM_CUDA(cudaMemcpyAsync(d_symbols, sym, 2 * n, cudaMemcpyDeviceToDevice, s));
  return check_status(sc, s);
}

void bm_release_workspace(void* stream) {
  std::lock_guard<std::mutex> g(g_ws_mu);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (stream == nullptr || it->first.second == s) {
      int cur = 0;
      cudaGetDevice(&cur);
      cudaSetDevice(it->second.dev);
      cudaStreamSynchronize(it->first.second);
      if (it->second.d) cudaFree(it->second.d);
      if (it->second.h) cudaFreeHost(it->second.h);
      if (it->second.aux) {
        cudaStreamSynchronize(it->second.aux);
        cudaStreamDestroy(it->second.aux);
        cudaEventDestroy(it->second.ev_fork);
        cudaEventDestroy(it->second.ev_join);
      }
      cudaSetDevice(cur);
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
}

}  // extern "C"

// ===========================================================================
// Allocation-free Huffman encoding (no cudaMalloc, no pinned host buffer)
// ===========================================================================
namespace bm {
namespace {

// Scratch of bm_huffman_encode_noalloc: one array per device, for the life of
// the process, shared by every call.
constexpr size_t kNoAllocBytes = size_t(1) << 20;     // 1 MiB
constexpr unsigned long long kNoAllocMaxChunks = 16384;
constexpr int kNoAllocMaxDict = 8192;  // at most this many present symbols: the codebook stays in shared memory
static_assert(kNoAllocMaxDict <= kEncWinSmall, "the encoder's window must hold the whole dictionary");
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_addr;  // device -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device.  In host code
// the array's name is only a stand-in, so the address is looked up once per
// device, with that device current, and cached.
bm_status noalloc_scratch(void** out) {
  int dev = 0;
  BM_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> g(g_noalloc_mu);
  auto it = g_noalloc_addr.find(dev);
  if (it != g_noalloc_addr.end()) {
    *out = it->second;
    return BM_OK;
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return fail(BM_ERR_CUDA, std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
  g_noalloc_addr[dev] = p;
  *out = p;
  return BM_OK;
}

}  // namespace
}  // namespace bm

extern "C" bm_status bm_huffman_encode_noalloc(const uint16_t* d_symbols, uint64_t n, int dict_size, int chunk_symbols,
                                               void* d_out, size_t out_capacity, uint64_t sizes_out[5], void* stream) {
  if (!d_symbols || !d_out || !sizes_out) return fail(BM_ERR_ARG, "NULL pointer argument");
  if (n == 0 || n >= (uint64_t(1) << 31)) return fail(BM_ERR_ARG, "symbol count must be in [1, 2^31)");
  if (dict_size < 2 || dict_size > kNoAllocMaxDict) return fail(BM_ERR_ARG, "dict_size must be in [2, 8192]");
  if (chunk_symbols < 64 || chunk_symbols > 2048 || chunk_symbols % 32) return fail(BM_ERR_ARG, "chunk_symbols");
  if (reinterpret_cast<uintptr_t>(d_out) % 8) return fail(BM_ERR_ARG, "output pointer must be 8-byte aligned");
  const unsigned long long nch = (n + chunk_symbols - 1) / chunk_symbols;
  if (nch > kNoAllocMaxChunks)
    return fail(BM_ERR_ARG, "more than 16384 chunks (n / chunk_symbols) do not fit the static scratch");
  const unsigned long long off_sp = pad8(4ull * nch);
  const unsigned long long off_cb = off_sp + pad8(2ull * (kSplits - 1) * nch);
  if (off_cb > out_capacity) return fail(BM_ERR_CAPACITY, "capacity below the chunk table");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the call ends with a device-to-host copy and a stream synchronisation,
  // neither of which a capturing stream allows
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  BM_CUDA(cudaStreamIsCapturing(s, &cap_st));
  if (cap_st != cudaStreamCaptureStatusNone)
    return fail(BM_ERR_ARG, "the stream is being captured: this call synchronises and cannot be captured");
  void* base = nullptr;
  if (bm_status st = noalloc_scratch(&base)) return st;
  Carver cv;
  cv.base = reinterpret_cast<unsigned char*>(base);
  Scalars* sc = cv.take<Scalars>(1);
  unsigned* hist = cv.take<unsigned>(dict_size);
  uint8_t* lens = cv.take<uint8_t>(dict_size);
  unsigned* codes = cv.take<unsigned>(dict_size);
  unsigned char* tickets = cv.take<unsigned char>(256 + 16ull * nch);
  unsigned* packed = cv.take<unsigned>(dict_size);
  if (cv.off > kNoAllocBytes) return fail(BM_ERR_ARG, "request does not fit the static scratch");
  uint8_t* out = reinterpret_cast<uint8_t*>(d_out);
  // the array keeps the previous call's contents: clear what must start at zero
  BM_CUDA(cudaMemsetAsync(sc, 0, sizeof(Scalars), s));
  BM_CUDA(cudaMemsetAsync(hist, 0, 4ull * dict_size, s));
  BM_CUDA(cudaMemsetAsync(tickets, 0, 256 + 16ull * nch, s));
  BM_CUDA(cudaMemsetAsync(out, 0, off_cb, s));
  hist_kernel<<<grid_for((int64_t)n, 256, 4), 256, 0, s>>>(d_symbols, n, dict_size, hist, sc);
  CodebookArgs ca{hist, dict_size, lens, codes, out, off_cb, out_capacity, sc, 0, nch, ~0ull, nullptr, packed};
  BM_CUDA(set_smem_once(codebook_kernel, (int)sizeof(CbSmem), g_cb_attr));
  codebook_kernel<<<1, kCbThreads, sizeof(CbSmem), s>>>(ca);
  FusedEncodeArgs ea{};
  ea.sym = d_symbols; ea.esc = nullptr; ea.n = n; ea.chunk = chunk_symbols; ea.lens = lens; ea.codes = codes;
  ea.dict = dict_size; ea.nch = nch; ea.ticket = reinterpret_cast<unsigned*>(tickets);
  ea.st = reinterpret_cast<unsigned long long*>(tickets + 256);
  ea.chunk_words = reinterpret_cast<unsigned*>(out); ea.out = out;
  ea.splits = reinterpret_cast<uint16_t*>(out + off_sp);
  ea.capacity = out_capacity; ea.sc = sc;
  ea.packed = packed;
  ea.win = kEncWinSmall;  // dict_size <= kNoAllocMaxDict = kEncWinSmall: every symbol in the window
  encode_fused_kernel<8, true, 0><<<grid_for((int64_t)nch * 32, 256, 4), 256, enc_smem<0>(kEncWinSmall), s>>>(ea);
  encode_finish_kernel<<<1, 32, 0, s>>>(~0ull, out_capacity, sc);
  zero_tail_kernel<<<1, 32, 0, s>>>(out, sc);
  g_launches.fetch_add(6);
  BM_CUDA(cudaGetLastError());
  Scalars hsc;
  BM_CUDA(cudaMemcpyAsync(&hsc, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s));
  BM_CUDA(cudaStreamSynchronize(s));
  if (hsc.status & ST_TIMEOUT) return fail(BM_ERR_CUDA, "encoder look-back wait timed out");
  if (hsc.status & ST_CORRUPT) return fail(BM_ERR_ARG, "a symbol is not below dict_size");
  if (hsc.status & (ST_RAW | ST_CAPACITY)) return fail(BM_ERR_CAPACITY, "output capacity too small");
  sizes_out[0] = hsc.codebook_bytes;
  sizes_out[1] = hsc.n_runs;
  sizes_out[2] = nch;
  sizes_out[3] = hsc.n_words;
  sizes_out[4] = pad8(hsc.off_bits + 4ull * hsc.n_words);
  return BM_OK;
}
