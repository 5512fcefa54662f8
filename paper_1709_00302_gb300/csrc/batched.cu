// Batched reductions: many independent matrices of uneven sizes, reduced in lockstep.
//
// Iteration t of every matrix still active runs in the same launches: one cluster panel
// launch (one thread-block cluster per matrix), then batched pack / streamed-product /
// reduce / rank-update launches of the split-precision engine whose per-matrix
// parameters come from device tables.  Matrices are ordered by their number of
// iterations, so the active set of iteration t is a prefix of that order.
//
// The host schedule is a deterministic function of the sizes and options: `plan`
// builds it, writes every parameter table into the workspace with one copy, and `run`
// rebuilds the same schedule and issues only kernel launches and memsets, so `run` can
// be captured into a CUDA graph and replayed.  sy2sb follows Section 2.1 (A1 update,
// X1 = A2 W, X2, X3, rank-2k update of A2); ge2gb follows Section 3.1 (left panel, E
// update, row panel, D update).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "driver.h"
#include "kernels.h"
#include "prof.h"
#include "split.h"

namespace bandred {

#define CK_RET(call)                                                \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call);     \
  } while (0)

namespace {

using split::PackParams;
using split::RankParams;
using split::ReduceParams;
using split::StreamParams;

constexpr size_t kAl = 256;
size_t al(size_t x) { return (x + kAl - 1) / kAl * kAl; }

enum LaunchType { kLPanel, kLPack, kLStream, kLReduce, kLRank };

struct Launch {
  LaunchType type;
  size_t off;    // byte offset of the parameter array in the table region
  int count;     // problems
  // launch shape
  int a = 0, b = 0;          // panel: C, Rp_max | stream: max_tiles, max_splits | rank: max_ti, max_tj
  int c = 0;                 // panel: bk_max | stream: BN
  int64_t big = 0;           // pack: max groups | reduce: max total
  // algorithmic flops and HBM bytes of all the launch's problems (profiler attribution;
  // the same counts as the single-matrix driver)
  double flops = 0.0, bytes = 0.0;
};

// Host side of a schedule: launch records plus the bytes of every parameter table.
struct Schedule {
  std::vector<Launch> launches;
  std::vector<unsigned char> table;
  bool fill = true;
  template <class T>
  size_t add(const std::vector<T>& v) {
    const size_t off = al(table.size());
    if (fill) {
      table.resize(off + sizeof(T) * v.size());
      std::memcpy(table.data() + off, v.data(), sizeof(T) * v.size());
    } else {
      table.resize(off + sizeof(T) * v.size());
    }
    return off;
  }
};

// Per-matrix pieces of the workspace.
struct Region {
  double *Y, *W, *X, *X2, *ZT, *P, *Yv, *Wv, *Pd;
  __nv_bfloat16 *wblob, *x2blob, *ablob, *bblob;
  size_t bytes;
};

struct Carve {
  char* base;
  size_t off;
  template <class T>
  T* take(size_t n) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += al(n * sizeof(T));
    return p;
  }
};

constexpr int kBatchSplits = 4;

int batch_b(const Options& o, int64_t w) { return (int)std::min<int64_t>(o.b > 0 ? o.b : std::min<int64_t>(w, 32), w); }

// Rows per CTA of the batched panels when the cluster size is not given: small enough
// that four CTAs share an SM (the FP64 work of one CTA overlaps the cluster barriers of
// the others), large enough that the barriers are few per row.
constexpr int kBatchPanelRows = 128;

// CTAs per problem (cluster size, a power of two <= 16) for panels of up to jmax x bkmax:
// `want` (the panel_ctas option) rounded up to a power of two, else the size that gives
// about kBatchPanelRows rows per CTA; raised until the slab fits in shared memory.
int cluster_size_for(int jmax, int bkmax, int want) {
  int C = 1;
  if (want > 0) {
    while (C < 16 && C < want) C *= 2;
  } else {
    while (C < 16 && (jmax + C - 1) / C > kBatchPanelRows) C *= 2;
  }
  while (C < 16 && panel_cluster_rows(jmax, bkmax, C) == 0) C *= 2;
  return C;
}

PackParams pack_b(const double* Bsrc, int64_t ldb, int K, int N, int S, __nv_bfloat16* out) {
  PackParams pp{};
  const int BN = split::stream_bn(N);
  pp.M1 = Bsrc;
  pp.ld1 = ldb;
  pp.K1 = K;
  pp.t1 = 1;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = N;
  pp.TR = BN;
  pp.TK = 32;
  pp.nrb = 1;
  pp.nkb = std::max(1, (K + 31) / 32);
  pp.S = S;
  pp.out = out;
  return pp;
}

PackParams pack_rows(const double* M1, int64_t ld1, int K1, const double* M2, int64_t ld2, int K2, int R, int Kr,
                     int S, __nv_bfloat16* out) {
  PackParams pp{};
  pp.M1 = M1;
  pp.ld1 = ld1;
  pp.K1 = K1;
  pp.t1 = 0;
  pp.M2 = M2;
  pp.ld2 = ld2;
  pp.K2 = K2;
  pp.t2 = 0;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = R;
  pp.TR = 128;
  pp.TK = 64;
  pp.nrb = (R + 127) / 128;
  pp.nkb = Kr / 64;
  pp.S = S;
  pp.out = out;
  return pp;
}

int64_t pack_groups(const PackParams& pp) { return (int64_t)pp.nrb * pp.nkb * pp.TR * (pp.TK / 8); }

// Collects the problems of one batched launch and appends the launch record.
struct Batcher {
  Schedule& S;
  int sms;
  int cluster;  // panel_ctas option: CTAs per problem of the panel launches (0 = auto)
  Batcher(Schedule& s, int n_sms, int cl) : S(s), sms(n_sms), cluster(cl) {}

  void packs(const std::vector<PackParams>& v) {
    if (v.empty()) return;
    Launch L{kLPack, S.add(v), (int)v.size()};
    for (const auto& p : v) {
      L.big = std::max(L.big, pack_groups(p));
      L.bytes += (8.0 + 2.0 * p.S) * p.R * (double)(p.K1 + p.K2);  // FP64 in, S bf16 slices out
    }
    S.launches.push_back(L);
  }
  void reduces(const std::vector<ReduceParams>& v) {
    if (v.empty()) return;
    Launch L{kLReduce, S.add(v), (int)v.size()};
    for (const auto& r : v) {
      L.big = std::max<int64_t>(L.big, (int64_t)r.M * r.N);
      L.bytes += 8.0 * r.M * (double)r.N * (r.splits + 1 + (r.beta != 0.0 ? 1 : 0));
    }
    S.launches.push_back(L);
  }
  // kt[q]: the reduction length of problem q before padding to Kr
  void ranks(const std::vector<RankParams>& v, const std::vector<int>& kt) {
    if (v.empty()) return;
    Launch L{kLRank, S.add(v), (int)v.size()};
    for (size_t q = 0; q < v.size(); ++q) {
      const RankParams& r = v[q];
      L.a = std::max(L.a, (r.M + 127) / 128);
      L.b = std::max(L.b, (std::min(r.N, r.col1) - 1) / 128 - r.tj0 + 1);
      const double nc = (double)(std::min(r.N, r.col1) - r.col0);
      // entries of C that change: the lower triangle (rows >= column) or the whole block
      const double entries = r.lower ? nc * r.M - nc * (nc - 1.0) / 2.0 : nc * r.M;
      L.flops += 2.0 * kt[q] * entries;
      L.bytes += 8.0 * (2.0 * entries + (double)(r.M + r.N) * kt[q]);
    }
    S.launches.push_back(L);
  }
  // Streamed products with a common split count chosen to fill the GPU.
  void streams(std::vector<StreamParams>& v, std::vector<ReduceParams>& red, int BN) {
    if (v.empty()) return;
    int64_t tiles = 0;
    int min_nkb = 1 << 30;
    for (const auto& p : v) {
      tiles += (p.M + 127) / 128;
      min_nkb = std::min(min_nkb, p.nkb);
    }
    int splits = 1;
    while (splits < kBatchSplits && tiles * splits < 2 * sms && min_nkb / (splits * 2) >= 2) splits *= 2;
    Launch L{kLStream, 0, (int)v.size()};
    L.c = BN;
    for (size_t q = 0; q < v.size(); ++q) {
      StreamParams& p = v[q];
      L.flops += 2.0 * p.M * (double)p.K * p.N;
      L.bytes += p.mode == split::kModeSymLower ? 8.0 * ((double)p.M * (p.M + 1) / 2.0 + 2.0 * p.M * (double)p.N)
                                                 : 8.0 * ((double)p.M * p.K + (double)p.K * p.N + (double)p.M * p.N);
      p.stages_per_split = (p.nkb + splits - 1) / splits;
      const int used = (p.nkb + p.stages_per_split - 1) / p.stages_per_split;
      red[q].splits = used;
      L.a = std::max(L.a, (p.M + 127) / 128);
      L.b = std::max(L.b, used);
    }
    L.off = S.add(v);
    S.launches.push_back(L);
    reduces(red);
  }
  void panels(const std::vector<PanelParams>& v) {
    if (v.empty()) return;
    int jmax = 0, bkmax = 0;
    for (const auto& p : v) {
      jmax = std::max(jmax, p.j);
      bkmax = std::max(bkmax, p.bk);
    }
    const int C = cluster_size_for(jmax, bkmax, cluster);
    std::vector<PanelParams> w = v;
    int Rpmax = 1;
    for (auto& p : w) {
      p.R = (p.j + C - 1) / C;
      p.Rp = p.R | 1;
      Rpmax = std::max(Rpmax, p.Rp);
    }
    Launch L{kLPanel, S.add(w), (int)w.size()};
    for (const auto& p : w) {  // Householder QR (2 j bk^2) and W = -Y T (j bk^2); 4 j bk doubles moved
      L.flops += 3.0 * p.j * (double)p.bk * p.bk;
      L.bytes += 32.0 * p.j * (double)p.bk;
    }
    L.a = C;
    L.b = Rpmax;
    L.c = bkmax;
    S.launches.push_back(L);
  }
};

PanelParams panel_of(double* A, int64_t rs, int64_t cs, int j, int bk, double* tau, double* Y, double* W, int64_t ldy,
                     const Options& o, int* status) {
  PanelParams p{};
  p.A = A;
  p.rs = rs;
  p.cs = cs;
  p.j = j;
  p.bk = bk;
  p.tau = tau;
  p.Y = Y;
  p.W = W;
  p.ldy = ldy;
  p.status = status;
  p.limit_ns = o.limit_ns;
  p.w_in_smem = true;
  p.w_fp32 = true;
  return p;
}

StreamParams stream_of(const double* A, int64_t lda, int mode, int M, int K, int N, const __nv_bfloat16* blob,
                       double* P, const Options& o, int* status) {
  StreamParams sp{};
  sp.A = A;
  sp.lda = lda;
  sp.mode = mode;
  sp.M = M;
  sp.K = K;
  sp.N = N;
  sp.Bblob = blob;
  sp.nkb = std::max(1, (K + 31) / 32);
  sp.stages_per_split = sp.nkb;
  sp.P = P;
  sp.ldp = M;
  sp.split_stride = (int64_t)M * N;
  sp.status = status;
  sp.limit_ns = o.limit_ns;
  return sp;
}

ReduceParams reduce_of(int M, int N, const double* P, double alpha, double beta, double* C, int64_t ldc) {
  return ReduceParams{M, N, 1, P, M, (int64_t)M * N, alpha, beta, C, ldc};
}

RankParams rank_of(const __nv_bfloat16* a, const __nv_bfloat16* b, int Kr, double* C, int64_t ldc, int M, int N,
                   int lower, const Options& o, int* status) {
  RankParams rp{};
  rp.Ablob = a;
  rp.Bblob = b;
  rp.Kr = Kr;
  rp.C = C;
  rp.ldc = ldc;
  rp.M = M;
  rp.N = N;
  rp.col0 = 0;
  rp.col1 = N;
  rp.lower = lower;
  rp.tj0 = 0;
  rp.alpha = 1.0;
  rp.status = status;
  rp.limit_ns = o.limit_ns;
  return rp;
}

// ------------------------------------------------------------------- sy2sb
struct SyMat {
  int64_t n, w, lda;
  int b, iters;
  double* A;
  double* tau;
  Region r;
};

Region carve_sy_region(Carve& c, int64_t n, int64_t w, int b, int S) {
  Region r{};
  const size_t start = c.off;
  const int64_t jmax = std::max<int64_t>(n - w, 1);
  const int BN = split::stream_bn(b);
  const int Kr = (2 * b + 63) / 64 * 64;
  r.Y = c.take<double>(jmax * b);
  r.W = c.take<double>(jmax * b);
  r.X = c.take<double>(jmax * b);
  r.X2 = c.take<double>((size_t)b * b);
  r.ZT = c.take<double>((size_t)w * b);
  r.P = c.take<double>((size_t)kBatchSplits * std::max<int64_t>(jmax, w) * BN + (size_t)kBatchSplits * BN * BN);
  r.wblob = c.take<__nv_bfloat16>(split::packed_bytes(BN, (int)jmax, BN, 32, S) / 2);
  r.x2blob = c.take<__nv_bfloat16>(split::packed_bytes(BN, b, BN, 32, S) / 2);
  r.ablob = c.take<__nv_bfloat16>(split::packed_bytes((int)jmax, Kr, 128, 64, S) / 2);
  r.bblob = c.take<__nv_bfloat16>(split::packed_bytes((int)std::max<int64_t>(jmax, w), Kr, 128, 64, S) / 2);
  r.bytes = c.off - start;
  return r;
}

void build_sy2sb(std::vector<SyMat>& mats, const Options& o, int S, int sms, int* status, Schedule& sch) {
  std::vector<int> order(mats.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mats[a].iters > mats[b].iters; });
  const int tmax = mats.empty() ? 0 : mats[order[0]].iters;
  Batcher B(sch, sms, o.panel_ctas);
  for (int t = 0; t < tmax; ++t) {
    std::vector<int> act;
    for (int q : order)
      if (mats[q].iters > t) act.push_back(q);
    // group by BN so that one stream launch has one tile shape
    std::vector<PanelParams> pan;
    for (int q : act) {
      SyMat& M = mats[q];
      const int64_t k = (int64_t)t * M.b;
      const int bk = (int)std::min<int64_t>(M.b, M.n - M.w - 1 - k);
      const int64_t r0 = k + M.w;
      const int j = (int)(M.n - r0);
      pan.push_back(panel_of(M.A + r0 + k * M.lda, 1, M.lda, j, bk, M.tau + k, M.r.Y, M.r.W, M.n - M.w, o, status));
    }
    B.panels(pan);
    for (int BN : {32, 64, 128}) {
      std::vector<int> g;
      for (int q : act)
        if (split::stream_bn(mats[q].b) == BN) g.push_back(q);
      if (g.empty()) continue;
      std::vector<PackParams> pk;
      std::vector<StreamParams> st;
      std::vector<ReduceParams> rd;
      auto geo = [&](const SyMat& M, int& bk, int64_t& k, int& j) {
        k = (int64_t)t * M.b;
        bk = (int)std::min<int64_t>(M.b, M.n - M.w - 1 - k);
        j = (int)(M.n - k - M.w);
      };
      for (int q : g) {  // W packed as the B operand of every streamed product with W
        const SyMat& M = mats[q];
        int bk, j;
        int64_t k;
        geo(M, bk, k, j);
        pk.push_back(pack_b(M.r.W, M.n - M.w, j, bk, S, M.r.wblob));
      }
      B.packs(pk);
      // A1 update (when the panel is narrower than w): Z^T = A1^T W, A1 += Y Z
      {
        std::vector<StreamParams> st1;
        std::vector<ReduceParams> rd1;
        std::vector<PackParams> pa, pb;
        std::vector<RankParams> rk;
        std::vector<int> kt;
        for (int q : g) {
          const SyMat& M = mats[q];
          int bk, j;
          int64_t k;
          geo(M, bk, k, j);
          const int na = (int)(M.w - bk);
          if (na <= 0) continue;
          double* A1 = M.A + (k + M.w) + (k + bk) * M.lda;
          st1.push_back(stream_of(A1, M.lda, split::kModeTrans, na, j, bk, M.r.wblob, M.r.P, o, status));
          rd1.push_back(reduce_of(na, bk, M.r.P, 1.0, 0.0, M.r.ZT, M.w));
          const int Kr = (bk + 63) / 64 * 64;
          pa.push_back(pack_rows(M.r.Y, M.n - M.w, bk, nullptr, 0, 0, j, Kr, S, M.r.ablob));
          pb.push_back(pack_rows(M.r.ZT, M.w, bk, nullptr, 0, 0, na, Kr, S, M.r.bblob));
          rk.push_back(rank_of(M.r.ablob, M.r.bblob, Kr, A1, M.lda, j, na, 0, o, status));
          kt.push_back(bk);
        }
        B.streams(st1, rd1, BN);
        B.packs(pa);
        B.packs(pb);
        B.ranks(rk, kt);
      }
      // X1 = A2 W
      for (int q : g) {
        const SyMat& M = mats[q];
        int bk, j;
        int64_t k;
        geo(M, bk, k, j);
        double* A2 = M.A + (k + M.w) * (1 + M.lda);
        st.push_back(stream_of(A2, M.lda, split::kModeSymLower, j, j, bk, M.r.wblob, M.r.P, o, status));
        rd.push_back(reduce_of(j, bk, M.r.P, 1.0, 0.0, M.r.X, M.n - M.w));
      }
      B.streams(st, rd, BN);
      // X2 = X1^T W / 2
      st.clear();
      rd.clear();
      for (int q : g) {
        const SyMat& M = mats[q];
        int bk, j;
        int64_t k;
        geo(M, bk, k, j);
        st.push_back(stream_of(M.r.X, M.n - M.w, split::kModeTrans, bk, j, bk, M.r.wblob, M.r.P, o, status));
        rd.push_back(reduce_of(bk, bk, M.r.P, 0.5, 0.0, M.r.X2, bk));
      }
      B.streams(st, rd, BN);
      // X3 = X1 + Y X2
      pk.clear();
      st.clear();
      rd.clear();
      for (int q : g) {
        const SyMat& M = mats[q];
        int bk, j;
        int64_t k;
        geo(M, bk, k, j);
        pk.push_back(pack_b(M.r.X2, bk, bk, bk, S, M.r.x2blob));
        st.push_back(stream_of(M.r.Y, M.n - M.w, split::kModePlain, j, bk, bk, M.r.x2blob, M.r.P, o, status));
        rd.push_back(reduce_of(j, bk, M.r.P, 1.0, 1.0, M.r.X, M.n - M.w));
      }
      B.packs(pk);
      B.streams(st, rd, BN);
      // A2 += X3 Y^T + Y X3^T (lower)
      std::vector<PackParams> pa, pb;
      std::vector<RankParams> rk;
      std::vector<int> kt;
      for (int q : g) {
        const SyMat& M = mats[q];
        int bk, j;
        int64_t k;
        geo(M, bk, k, j);
        const int Kr = (2 * bk + 63) / 64 * 64;
        const int64_t ld = M.n - M.w;
        pa.push_back(pack_rows(M.r.X, ld, bk, M.r.Y, ld, bk, j, Kr, S, M.r.ablob));
        pb.push_back(pack_rows(M.r.Y, ld, bk, M.r.X, ld, bk, j, Kr, S, M.r.bblob));
        double* A2 = M.A + (k + M.w) * (1 + M.lda);
        rk.push_back(rank_of(M.r.ablob, M.r.bblob, Kr, A2, M.lda, j, j, 1, o, status));
        kt.push_back(2 * bk);
      }
      B.packs(pa);
      B.packs(pb);
      B.ranks(rk, kt);
    }
  }
}

// ------------------------------------------------------------------- ge2gb
struct GeMat {
  int64_t m, n, w, lda;
  int b, iters;
  double *A, *tauq, *taup;
  Region r;
};

Region carve_ge_region(Carve& c, int64_t m, int64_t n, int b, int S) {
  Region r{};
  const size_t start = c.off;
  const int64_t big = std::max<int64_t>(std::max(m, n), 1);
  const int BN = split::stream_bn(b);
  const int Kr = (b + 63) / 64 * 64;
  r.Y = c.take<double>(std::max<int64_t>(m, 1) * b);
  r.W = c.take<double>(std::max<int64_t>(m, 1) * b);
  r.Yv = c.take<double>(std::max<int64_t>(n, 1) * b);
  r.Wv = c.take<double>(std::max<int64_t>(n, 1) * b);
  r.ZT = c.take<double>(std::max<int64_t>(n, 1) * b);
  r.Pd = c.take<double>(std::max<int64_t>(m, 1) * b);
  r.P = c.take<double>((size_t)kBatchSplits * big * BN);
  r.wblob = c.take<__nv_bfloat16>(split::packed_bytes(BN, (int)big, BN, 32, S) / 2);
  r.ablob = c.take<__nv_bfloat16>(split::packed_bytes((int)big, Kr, 128, 64, S) / 2);
  r.bblob = c.take<__nv_bfloat16>(split::packed_bytes((int)big, Kr, 128, 64, S) / 2);
  r.bytes = c.off - start;
  return r;
}

void build_ge2gb(std::vector<GeMat>& mats, const Options& o, int S, int sms, int* status, Schedule& sch) {
  std::vector<int> order(mats.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return mats[a].iters > mats[b].iters; });
  const int tmax = mats.empty() ? 0 : mats[order[0]].iters;
  Batcher B(sch, sms, o.panel_ctas);
  for (int t = 0; t < tmax; ++t) {
    std::vector<int> act;
    for (int q : order)
      if (mats[q].iters > t) act.push_back(q);
    std::vector<PanelParams> pan;
    for (int q : act) {
      GeMat& M = mats[q];
      const int64_t k = (int64_t)t * M.b;
      const int bk = (int)std::min<int64_t>(M.b, M.n - k);
      pan.push_back(panel_of(M.A + k + k * M.lda, 1, M.lda, (int)(M.m - k), bk, M.tauq + k, M.r.Y, M.r.W, M.m, o, status));
    }
    B.panels(pan);
    for (int BN : {32, 64, 128}) {
      std::vector<int> g;
      for (int q : act)
        if (split::stream_bn(mats[q].b) == BN) g.push_back(q);
      if (g.empty()) continue;
      // left update E += Y_U (W_U^T E)
      std::vector<PackParams> pk, pa, pb;
      std::vector<StreamParams> st;
      std::vector<ReduceParams> rd;
      std::vector<RankParams> rk;
      std::vector<int> kt;
      for (int q : g) {
        const GeMat& M = mats[q];
        const int64_t k = (int64_t)t * M.b;
        const int bk = (int)std::min<int64_t>(M.b, M.n - k);
        const int j = (int)(M.m - k);
        const int nc = (int)(M.n - k - bk);
        if (nc <= 0) continue;
        double* E = M.A + k + (k + bk) * M.lda;
        pk.push_back(pack_b(M.r.W, M.m, j, bk, S, M.r.wblob));
        st.push_back(stream_of(E, M.lda, split::kModeTrans, nc, j, bk, M.r.wblob, M.r.P, o, status));
        rd.push_back(reduce_of(nc, bk, M.r.P, 1.0, 0.0, M.r.ZT, M.n));
        const int Kr = (bk + 63) / 64 * 64;
        pa.push_back(pack_rows(M.r.Y, M.m, bk, nullptr, 0, 0, j, Kr, S, M.r.ablob));
        pb.push_back(pack_rows(M.r.ZT, M.n, bk, nullptr, 0, 0, nc, Kr, S, M.r.bblob));
        rk.push_back(rank_of(M.r.ablob, M.r.bblob, Kr, E, M.lda, j, nc, 0, o, status));
        kt.push_back(bk);
      }
      B.packs(pk);
      B.streams(st, rd, BN);
      B.packs(pa);
      B.packs(pb);
      B.ranks(rk, kt);
    }
    // row panels
    pan.clear();
    for (int q : act) {
      GeMat& M = mats[q];
      const int64_t k = (int64_t)t * M.b;
      const int bk = (int)std::min<int64_t>(M.b, M.n - k);
      const int64_t bkr = std::min<int64_t>(bk, M.n - M.w - 1 - k);
      if (bkr <= 0) continue;
      pan.push_back(panel_of(M.A + k + (k + M.w) * M.lda, M.lda, 1, (int)(M.n - k - M.w), (int)bkr, M.taup + k, M.r.Yv,
                             M.r.Wv, M.n, o, status));
    }
    B.panels(pan);
    for (int BN : {32, 64, 128}) {
      std::vector<PackParams> pk, pa, pb;
      std::vector<StreamParams> st;
      std::vector<ReduceParams> rd;
      std::vector<RankParams> rk;
      std::vector<int> kt;
      for (int q : act) {
        const GeMat& M = mats[q];
        if (split::stream_bn(M.b) != BN) continue;
        const int64_t k = (int64_t)t * M.b;
        const int bk = (int)std::min<int64_t>(M.b, M.n - k);
        const int bkr = (int)std::min<int64_t>(bk, M.n - M.w - 1 - k);
        if (bkr <= 0) continue;
        const int jr = (int)(M.n - k - M.w);
        const int nrow = (int)(M.m - k - bkr);
        if (nrow <= 0) continue;
        double* D = M.A + (k + bkr) + (k + M.w) * M.lda;
        pk.push_back(pack_b(M.r.Wv, M.n, jr, bkr, S, M.r.wblob));
        st.push_back(stream_of(D, M.lda, split::kModePlain, nrow, jr, bkr, M.r.wblob, M.r.P, o, status));
        rd.push_back(reduce_of(nrow, bkr, M.r.P, 1.0, 0.0, M.r.Pd, M.m));
        const int Kr = (bkr + 63) / 64 * 64;
        pa.push_back(pack_rows(M.r.Pd, M.m, bkr, nullptr, 0, 0, nrow, Kr, S, M.r.ablob));
        pb.push_back(pack_rows(M.r.Yv, M.n, bkr, nullptr, 0, 0, jr, Kr, S, M.r.bblob));
        rk.push_back(rank_of(M.r.ablob, M.r.bblob, Kr, D, M.lda, nrow, jr, 0, o, status));
        kt.push_back(bkr);
      }
      B.packs(pk);
      B.streams(st, rd, BN);
      B.packs(pa);
      B.packs(pb);
      B.ranks(rk, kt);
    }
  }
}

// Launch a schedule whose tables live at `table` (device).
int launch_schedule(const Schedule& sch, const unsigned char* table, int S, cudaStream_t s) {
  for (const Launch& L : sch.launches) {
    const void* p = table + L.off;
    cudaError_t e = cudaSuccess;
    switch (L.type) {
      case kLPanel: {
        prof::Scope sc(prof::kPanel, s, L.flops, L.bytes);
        e = launch_panel_cluster(nullptr, static_cast<const PanelParams*>(p), L.count, L.a, L.b, L.c, s);
        break;
      }
      case kLPack: {
        prof::Scope sc(prof::kConvert, s, L.flops, L.bytes);
        e = split::pack_batched(static_cast<const PackParams*>(p), L.count, L.big, s);
        break;
      }
      case kLStream: {
        prof::Scope sc(prof::kSymm, s, L.flops, L.bytes);
        e = split::stream_gemm_batched(static_cast<const StreamParams*>(p), L.count, S, L.c, L.a, L.b, s);
        break;
      }
      case kLReduce: {
        prof::Scope sc(prof::kSplitReduce, s, L.flops, L.bytes);
        e = split::reduce_batched(static_cast<const ReduceParams*>(p), L.count, L.big, s);
        break;
      }
      case kLRank: {
        prof::Scope sc(prof::kSyr2k, s, L.flops, L.bytes);
        e = split::rank_update_batched(static_cast<const RankParams*>(p), L.count, S, L.a, L.b, s);
        break;
      }
    }
    if (e != cudaSuccess) return record_cuda_error(e, "batched launch");
  }
  return 0;
}

int sms_of_current() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Workspace: [status | table | regions].  Returns the total bytes; fills `sch` and the
// matrices' regions when base != nullptr.
template <class Mat, class CarveFn, class BuildFn>
size_t layout(std::vector<Mat>& mats, const Options& o, char* base, bool fill, CarveFn carve_region, BuildFn build,
              Schedule& sch, int** status_out) {
  const int S = split::slices_of(o.precision);
  // regions first (sizes do not depend on the schedule), then the table
  Carve c{base, 0};
  int* status = c.take<int>(64);
  const size_t regions_start = c.off;
  for (auto& M : mats) M.r = carve_region(c, M);
  const size_t table_off = c.off;
  sch.fill = fill;
  build(mats, o, S, sms_of_current(), status, sch);
  if (status_out) *status_out = status;
  (void)regions_start;
  return table_off + al(sch.table.size());
}

bool batched_opts_ok(const Options& o) { return o.precision == BANDRED_BF16X3 || o.precision == BANDRED_BF16X6; }

}  // namespace

// ------------------------------------------------------------------- entry points
int sy2sb_batched(int count, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda,
                  double* const* tau, const Options& o, void* work, size_t work_bytes, int* dev_status,
                  cudaStream_t s, int mode) {
  if (!batched_opts_ok(o)) return BANDRED_ERR_UNSUPPORTED;
  std::vector<SyMat> mats(count);
  for (int q = 0; q < count; ++q) {
    SyMat& M = mats[q];
    M.n = n[q];
    M.w = w[q];
    M.lda = lda ? lda[q] : n[q];
    M.b = batch_b(o, M.w);
    M.A = A ? A[q] : nullptr;
    M.tau = tau ? tau[q] : nullptr;
    M.iters = M.n - M.w - 2 >= 0 ? (int)((M.n - M.w - 2) / M.b + 1) : 0;
  }
  const int S = split::slices_of(o.precision);
  auto carve = [&](Carve& c, const SyMat& M) { return carve_sy_region(c, M.n, M.w, M.b, S); };
  Schedule sch;
  int* status = nullptr;
  const size_t bytes = layout(mats, o, static_cast<char*>(work), mode == 1, carve, build_sy2sb, sch, &status);
  if (work_bytes < bytes) return BANDRED_ERR_WORKSPACE;
  const unsigned char* table = static_cast<unsigned char*>(work) + (bytes - al(sch.table.size()));
  if (mode == 1) {  // plan: tau cleared once, tables uploaded
    for (int q = 0; q < count; ++q)
      if (mats[q].n - mats[q].w > 0 && tau[q])
        CK_RET(cudaMemsetAsync(tau[q], 0, sizeof(double) * (mats[q].n - mats[q].w), s));
    CK_RET(cudaMemcpyAsync(const_cast<unsigned char*>(table), sch.table.data(), sch.table.size(),
                           cudaMemcpyHostToDevice, s));
    return 0;
  }
  // The tables carry the workspace's status word; it is cleared here and copied to the
  // caller's status word after the launches.
  CK_RET(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (int rc = launch_schedule(sch, table, S, s)) return rc;
  if (dev_status) CK_RET(cudaMemcpyAsync(dev_status, status, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return 0;
}

size_t sy2sb_batched_workspace(int count, const int64_t* n, const int64_t* w, const Options& o) {
  if (!batched_opts_ok(o)) return 0;
  std::vector<SyMat> mats(count);
  for (int q = 0; q < count; ++q) {
    mats[q].n = n[q];
    mats[q].w = w[q];
    mats[q].lda = n[q];
    mats[q].b = batch_b(o, w[q]);
    mats[q].iters = n[q] - w[q] - 2 >= 0 ? (int)((n[q] - w[q] - 2) / mats[q].b + 1) : 0;
  }
  const int S = split::slices_of(o.precision);
  auto carve = [&](Carve& c, const SyMat& M) { return carve_sy_region(c, M.n, M.w, M.b, S); };
  Schedule sch;
  return layout(mats, o, nullptr, false, carve, build_sy2sb, sch, nullptr);
}

int ge2gb_batched(int count, const int64_t* m, const int64_t* n, const int64_t* w, double* const* A,
                  const int64_t* lda, double* const* tauq, double* const* taup, const Options& o, void* work,
                  size_t work_bytes, int* dev_status, cudaStream_t s, int mode) {
  if (!batched_opts_ok(o)) return BANDRED_ERR_UNSUPPORTED;
  std::vector<GeMat> mats(count);
  for (int q = 0; q < count; ++q) {
    GeMat& M = mats[q];
    M.m = m[q];
    M.n = n[q];
    M.w = w[q];
    M.lda = lda ? lda[q] : m[q];
    M.b = batch_b(o, M.w);
    M.A = A ? A[q] : nullptr;
    M.tauq = tauq ? tauq[q] : nullptr;
    M.taup = taup ? taup[q] : nullptr;
    M.iters = M.n > 0 ? (int)((M.n + M.b - 1) / M.b) : 0;
  }
  const int S = split::slices_of(o.precision);
  auto carve = [&](Carve& c, const GeMat& M) { return carve_ge_region(c, M.m, M.n, M.b, S); };
  Schedule sch;
  int* status = nullptr;
  const size_t bytes = layout(mats, o, static_cast<char*>(work), mode == 1, carve, build_ge2gb, sch, &status);
  if (work_bytes < bytes) return BANDRED_ERR_WORKSPACE;
  const unsigned char* table = static_cast<unsigned char*>(work) + (bytes - al(sch.table.size()));
  if (mode == 1) {
    for (int q = 0; q < count; ++q) {
      if (mats[q].n > 0 && tauq[q]) CK_RET(cudaMemsetAsync(tauq[q], 0, sizeof(double) * mats[q].n, s));
      if (mats[q].n - mats[q].w > 0 && taup[q])
        CK_RET(cudaMemsetAsync(taup[q], 0, sizeof(double) * (mats[q].n - mats[q].w), s));
    }
    CK_RET(cudaMemcpyAsync(const_cast<unsigned char*>(table), sch.table.data(), sch.table.size(),
                           cudaMemcpyHostToDevice, s));
    return 0;
  }
  // The tables carry the workspace's status word; it is cleared here and copied to the
  // caller's status word after the launches.
  CK_RET(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (int rc = launch_schedule(sch, table, S, s)) return rc;
  if (dev_status) CK_RET(cudaMemcpyAsync(dev_status, status, sizeof(int), cudaMemcpyDeviceToDevice, s));
  return 0;
}

size_t ge2gb_batched_workspace(int count, const int64_t* m, const int64_t* n, const int64_t* w, const Options& o) {
  if (!batched_opts_ok(o)) return 0;
  std::vector<GeMat> mats(count);
  for (int q = 0; q < count; ++q) {
    mats[q].m = m[q];
    mats[q].n = n[q];
    mats[q].w = w[q];
    mats[q].lda = m[q];
    mats[q].b = batch_b(o, w[q]);
    mats[q].iters = n[q] > 0 ? (int)((n[q] + mats[q].b - 1) / mats[q].b) : 0;
  }
  const int S = split::slices_of(o.precision);
  auto carve = [&](Carve& c, const GeMat& M) { return carve_ge_region(c, M.m, M.n, M.b, S); };
  Schedule sch;
  return layout(mats, o, nullptr, false, carve, build_ge2gb, sch, nullptr);
}

}  // namespace bandred

// ------------------------------------------------------------------- C ABI
namespace {

int check_batch_common(int count, const bandred_opts* opts, int64_t wmax, bandred::Options* o) {
  if (count < 0) return -1;
  if (bandred::resolve_options(opts, std::max<int64_t>(wmax, 1), o) != 0) return -7;
  return 0;
}

bool device_ok(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int check_sy(int count, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda, double* const* tau,
             const bandred_opts* opts, bandred::Options* o) {
  if (count < 0) return -1;
  if (count > 0 && (!n || !w || !A || !tau)) return -2;
  int64_t wmax = 1;
  for (int q = 0; q < count; ++q) {
    if (n[q] < 0) return -2;
    if (w[q] < 1) return -3;
    if (n[q] > 0 && !A[q]) return -4;
    if ((lda ? lda[q] : n[q]) < std::max<int64_t>(1, n[q])) return -5;
    if (n[q] - w[q] > 0 && !tau[q]) return -6;
    wmax = std::max(wmax, w[q]);
  }
  return check_batch_common(count, opts, wmax, o);
}

int check_ge(int count, const int64_t* m, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda,
             double* const* tauq, double* const* taup, const bandred_opts* opts, bandred::Options* o) {
  if (count < 0) return -1;
  if (count > 0 && (!m || !n || !w || !A || !tauq || !taup)) return -2;
  int64_t wmax = 1;
  for (int q = 0; q < count; ++q) {
    if (m[q] < 0 || n[q] < 0 || n[q] > m[q]) return -3;
    if (w[q] < 1) return -4;
    if (n[q] > 0 && !A[q]) return -5;
    if ((lda ? lda[q] : m[q]) < std::max<int64_t>(1, m[q])) return -6;
    if ((n[q] > 0 && !tauq[q]) || (n[q] - w[q] > 0 && !taup[q])) return -7;
    wmax = std::max(wmax, w[q]);
  }
  return check_batch_common(count, opts, wmax, o) == -7 ? -9 : 0;
}

}  // namespace

extern "C" {

size_t bandred_sy2sb_batched_workspace(int count, const int64_t* n, const int64_t* w, const bandred_opts* opts) {
  bandred::Options o;
  if (count < 0 || (count > 0 && (!n || !w))) return 0;
  int64_t wmax = 1;
  for (int q = 0; q < count; ++q) wmax = std::max(wmax, w[q]);
  if (bandred::resolve_options(opts, wmax, &o) != 0) return 0;
  return bandred::sy2sb_batched_workspace(count, n, w, o);
}

int bandred_sy2sb_batched_plan(int count, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda,
                               double* const* tau, const bandred_opts* opts, void* work, size_t work_bytes,
                               cudaStream_t stream) {
  bandred::Options o;
  if (int rc = check_sy(count, n, w, A, lda, tau, opts, &o)) return rc;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) || !device_ok(work)) return -8;
  return bandred::sy2sb_batched(count, n, w, A, lda, tau, o, work, work_bytes, nullptr, stream, 1);
}

int bandred_sy2sb_batched_run(int count, const int64_t* n, const int64_t* w, double* const* A, const int64_t* lda,
                              double* const* tau, const bandred_opts* opts, void* work, size_t work_bytes,
                              int* dev_status, cudaStream_t stream) {
  bandred::Options o;
  if (int rc = check_sy(count, n, w, A, lda, tau, opts, &o)) return rc;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u)) return -8;
  return bandred::sy2sb_batched(count, n, w, A, lda, tau, o, work, work_bytes, dev_status, stream, 2);
}

size_t bandred_ge2gb_batched_workspace(int count, const int64_t* m, const int64_t* n, const int64_t* w,
                                       const bandred_opts* opts) {
  bandred::Options o;
  if (count < 0 || (count > 0 && (!m || !n || !w))) return 0;
  int64_t wmax = 1;
  for (int q = 0; q < count; ++q) wmax = std::max(wmax, w[q]);
  if (bandred::resolve_options(opts, wmax, &o) != 0) return 0;
  return bandred::ge2gb_batched_workspace(count, m, n, w, o);
}

int bandred_ge2gb_batched_plan(int count, const int64_t* m, const int64_t* n, const int64_t* w, double* const* A,
                               const int64_t* lda, double* const* tauq, double* const* taup, const bandred_opts* opts,
                               void* work, size_t work_bytes, cudaStream_t stream) {
  bandred::Options o;
  if (int rc = check_ge(count, m, n, w, A, lda, tauq, taup, opts, &o)) return rc;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u) || !device_ok(work)) return -10;
  return bandred::ge2gb_batched(count, m, n, w, A, lda, tauq, taup, o, work, work_bytes, nullptr, stream, 1);
}

int bandred_ge2gb_batched_run(int count, const int64_t* m, const int64_t* n, const int64_t* w, double* const* A,
                              const int64_t* lda, double* const* tauq, double* const* taup, const bandred_opts* opts,
                              void* work, size_t work_bytes, int* dev_status, cudaStream_t stream) {
  bandred::Options o;
  if (int rc = check_ge(count, m, n, w, A, lda, tauq, taup, opts, &o)) return rc;
  if (!work || (reinterpret_cast<uintptr_t>(work) & 255u)) return -10;
  return bandred::ge2gb_batched(count, m, n, w, A, lda, tauq, taup, o, work, work_bytes, dev_status, stream, 2);
}

}  // extern "C"
