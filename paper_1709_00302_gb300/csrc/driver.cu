// Host side of the C ABI declared in include/bandred.h: argument checks, workspace
// layout, and the blocked right-looking loops of Section 2.1 (sy2sb) and Section 3.1
// (ge2gb), with the look-ahead of Sections 2.2 and 3.2 expressed as two CUDA streams:
// a high-priority stream runs the part of the trailing update that feeds the next panel
// and then factors that panel, while the default-priority stream updates the rest.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "driver.h"
#include "ozaki.h"
#include "kernels.h"
#include "prof.h"
#include "split.h"

namespace bandred {

namespace {

constexpr size_t kAlign = 256;
constexpr int kMinPanelRows = 16;
constexpr int kClusterMax = 16;    // CTAs of a cluster panel
constexpr int kClusterRows = 32;   // a panel of at most kClusterMax * kClusterRows rows may use a cluster
constexpr int kClusterMinRows = 16;  // rows per cluster CTA the cluster size aims at (more CTAs: less FP64 each)
// The single-matrix reductions take the grid panel at every size by default: measured on
// GB300 its paired steps (two reflectors per grid reduction) beat the cluster panel's one
// reflector per cluster barrier on the last panels (j <= 512: about 0.2 against 0.28-0.3
// ms), and a 16-CTA cluster needs 16 free SMs in one GPC, which the capped update beside
// it rarely leaves.  The cluster panel is the batched path's, one cluster per matrix, and
// the single-matrix reductions' with opts->panel_group = 1.
static bool cluster_panels(const Options& o) { return o.panel_group == 1; }
constexpr int kMaxSplits = 128;
constexpr int kSmallSplits = 32;       // split-K of the FP64 products with a b-wide output
constexpr int kMaxStreamSplits = 8;    // split-K of the streamed X1 = A2 W product
constexpr int kMaxSmallSplits = 256;   // split-K of the b x b product X1^T W

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

thread_local char g_last_error[512] = "";

struct DeviceInfo {
  int sms = 0;
};

constexpr int kMaxDevices = 64;  // devices a process may use with this library

DeviceInfo& device_info(int dev) {
  static std::mutex mu;
  static DeviceInfo info[kMaxDevices];
  static DeviceInfo other;  // beyond kMaxDevices: asked every time
  std::lock_guard<std::mutex> lock(mu);
  DeviceInfo& d = (dev >= 0 && dev < kMaxDevices) ? info[dev] : other;
  if (d.sms == 0 || &d == &other) cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
  return d;
}

// Carves a workspace into 256-byte aligned pieces; with base == nullptr it only sizes.
struct Carver {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align_up(count * sizeof(T));
    return p;
  }
};

// Panel CTAs per SM (two per SM were measured slower: the per-step barrier and scalar
// chain do not shrink, while the CTAs compete for the FP64 pipe).
constexpr int kPanelCtasPerSm = 1;

int panel_max_ctas(int sms, const Options& o) {
  if (o.panel_ctas > 0) return std::min(o.panel_ctas, kPanelCtasPerSm * sms);
  return kPanelCtasPerSm * sms;
}

int choose_splits(int M, int N, int K, size_t capacity_doubles, int sms) {
  const int tiles = ((M + 63) / 64) * ((N + 63) / 64);
  if (tiles >= sms || K <= 512) return 1;
  int s = std::min(kMaxSplits, std::max(1, (2 * sms) / std::max(tiles, 1)));
  s = std::min(s, std::max(1, K / 256));
  while (s > 1 && (size_t)s * M * N > capacity_doubles) --s;
  return s;
}

// Algorithmic flop and HBM-byte counts attributed to each kernel class by the profiler.
// Householder QR of a j x bk panel (2 j bk^2) plus the W = -Y T build (j bk^2); the panel
// is read and written once and Y, W are written once.
double panel_flops(double j, double bk) { return 3.0 * j * bk * bk; }
double panel_bytes(double j, double bk) { return 8.0 * 4.0 * j * bk; }
// X1 = A2 W over the lower triangle of A2 (read once) with W read and X1 written once.
double symm_flops(double j, double bk) { return 2.0 * j * j * bk; }
double symm_bytes(double j, double bk) { return 8.0 * (j * (j + 1) / 2 + 2.0 * j * bk); }
// A2 += X3 Y^T + Y X3^T on the lower triangle of columns [c0, c1) (read and written once).
double lower_entries(double j, double c0, double c1) { return (c1 - c0) * j - (c1 * (c1 - 1) - c0 * (c0 - 1)) / 2; }
double syr2k_flops(double j, double c0, double c1, double bk) { return 4.0 * bk * lower_entries(j, c0, c1); }
double syr2k_bytes(double j, double c0, double c1, double bk) {
  return 8.0 * (2.0 * lower_entries(j, c0, c1) + 2.0 * j * bk);
}

}  // namespace

int record_cuda_error(cudaError_t e, const char* what) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e),
                what);
  cudaGetLastError();  // clear a sticky launch error so that later calls can proceed
  return BANDRED_ERR_CUDA;
}

const char* last_cuda_error() { return g_last_error; }

// ---------------------------------------------------------------------------------
int resolve_options(const bandred_opts* in, int64_t w, Options* o) {
  bandred_opts d;
  bandred_default_opts(&d);
  if (in) d = *in;
  for (int r : d.reserved)
    if (r != 0) return -1;
  if (d.b == 0) d.b = (int)std::min<int64_t>(w, 64);
  if (d.b < 1 || d.b > w) return -1;
  if (d.lookahead < -1 || d.lookahead > 2) return -1;
  if (d.precision < 0 || d.precision > 3) return -1;
  if (d.panel_ctas < 0 || d.timeout_ms < 0) return -1;
  if (d.debug < 0 || d.debug > 1) return -1;
  if (d.panel_group != 0 && d.panel_group != 1 && d.panel_group != 2 && d.panel_group != 4) return -1;
  if (d.depth < 0 || d.depth > 2) return -1;
  o->b = d.b;
  o->lookahead = d.lookahead;
  o->precision = d.precision;
  o->slices = d.slices;
  o->panel_ctas = d.panel_ctas;
  o->limit_ns = (unsigned long long)(d.timeout_ms ? d.timeout_ms : 2000) * 1000000ull;
  o->debug = d.debug;
  o->panel_group = d.panel_group ? d.panel_group : 2;
  o->depth = d.depth ? d.depth : 1;
  return 0;
}

// Workspace of sy2sb (layout shared by sizing and carving).  Y and W are double-buffered:
// with look-ahead the next panel writes one pair while the current update reads the other.
// W of an Ozaki-precision panel as one tensor-core product W = Y Tn (Tn = -T from the
// panel's Gram coefficients), instead of the FP64 forward substitution.
struct PanelW {
  double* Tn;    // bk x bk
  char* oz;      // Ozaki buffers of a j x bk x bk product
  size_t oz_cap;
};

struct Sy2sbWs {
  double *Y[3], *W[3], *X, *X2;
  PanelW pw;
  double *Z[2], *splitk[2];  // FP64 small products; [1] belongs to the panel stream
  double *part, *rowbuf, *gram;
  GridSync* gs;
  // split-precision buffers
  __nv_bfloat16 *wblob, *x2blob, *ablob, *bblob;
  double* P;
  size_t P_cap;
  // Ozaki-scheme buffers: products (exponents, packed operands, split partials) and the
  // packed operands of the rank-2k update
  char *ozp, *ozr;
  size_t ozp_cap;
  int* weB;                // W's exponents and digits as the right operand of X1 = A2 W, kept
  __nv_bfloat16* wblobz;   // for X2 = X1^T W / 2 (the same right operand)
  int64_t ld;
  size_t splitk_cap;
  int* status;
  size_t bytes;
};

static bool is_split(const Options& o) { return o.precision == BANDRED_BF16X3 || o.precision == BANDRED_BF16X6; }

// Look-ahead of sy2sb (Section 2.2): 0 none, 1 Variant V1 (2b <= w: the next panel lies in
// A1), 2 Variant V2 (2b > w: it lies in A2).  Auto picks the variant the sizes allow.
static int sy2sb_variant(const Options& o, int64_t w) {
  int la = o.lookahead;
  if (la < 0) la = (2 * o.b > w) ? 2 : 1;
  if (la == 1 && 2 * o.b > w) la = 0;  // V1 needs 2b <= w
  if (la == 2 && 2 * o.b <= w) la = 1;
  return la;
}

// Depth 2 (the panel two iterations ahead) is open to V1 when 3b <= w: that panel's columns
// then lie in A1 of this iteration and of the next, so one-sided updates alone reach it.
static int sy2sb_depth(const Options& o, int64_t w) {
  return (o.depth == 2 && sy2sb_variant(o, w) == 1 && 3 * (int64_t)o.b <= w) ? 2 : 1;
}

static Sy2sbWs carve_sy2sb(void* work, int64_t n, int64_t w, const Options& o, int sms) {
  Carver c{static_cast<char*>(work)};
  Sy2sbWs ws{};
  const int64_t jmax = std::max<int64_t>(n - w, 1);
  const int64_t b = o.b;
  ws.ld = jmax;
  // Y/W: one pair per panel alive at once (1 without look-ahead, 2 at depth 1, 3 at depth
  // 2); the panel stream's product buffers exist only with look-ahead
  const int nbuf = o.lookahead == 0 ? 1 : 2;
  const int nyw = o.lookahead == 0 ? 1 : 1 + sy2sb_depth(o, w);
  for (int q = 0; q < 3; ++q) {
    ws.Y[q] = q < nyw ? c.take<double>(jmax * b) : ws.Y[0];
    ws.W[q] = q < nyw ? c.take<double>(jmax * b) : ws.W[0];
  }
  ws.X = c.take<double>(jmax * b);
  ws.X2 = c.take<double>(b * b);
  ws.splitk_cap = (size_t)kSmallSplits * b * std::max<int64_t>(w, b);
  for (int q = 0; q < 2; ++q) {
    ws.Z[q] = q < nbuf ? c.take<double>(b * std::max<int64_t>(w, 1)) : ws.Z[0];
    ws.splitk[q] = q < nbuf ? c.take<double>(ws.splitk_cap) : ws.splitk[0];
  }
  ws.rowbuf = c.take<double>(8 * (size_t)b);  // up to four rows per step, two steps
  ws.gram = c.take<double>((size_t)b * b);    // Gram coefficients of the panel (W formed after it)
  ws.gs = c.take<GridSync>(1);  // 256 bytes, immediately followed by the accumulators
  ws.part = c.take<double>((panel_sync_bytes((int)b) - 256) / sizeof(double));
  if (is_split(o)) {
    const int S = split::slices_of(o.precision);
    const int BN = split::stream_bn((int)b);
    const int Kr = (int)((2 * b + 63) / 64 * 64);
    ws.wblob = c.take<__nv_bfloat16>(split::packed_bytes(BN, (int)jmax, BN, 32, S) / 2);
    ws.x2blob = c.take<__nv_bfloat16>(split::packed_bytes(BN, (int)b, BN, 32, S) / 2);
    ws.ablob = c.take<__nv_bfloat16>(split::packed_bytes((int)jmax, Kr, 128, 64, S) / 2);
    ws.bblob = c.take<__nv_bfloat16>(split::packed_bytes((int)jmax, Kr, 128, 64, S) / 2);
    ws.P_cap = std::max<size_t>((size_t)kMaxStreamSplits * jmax * BN, (size_t)kMaxSmallSplits * BN * BN);
    ws.P = c.take<double>(ws.P_cap);
  }
  if (o.precision == BANDRED_OZAKI) {
    const int J = (int)jmax, B = (int)b;
    ws.ozp_cap = ozaki::bytes(J, B, J, ozaki::choose_splits(J, B, J, sms));
    ws.ozp = c.take<char>(ws.ozp_cap);
    ws.ozr = c.take<char>(ozaki::bytes(J, J, 2 * B, 1, false));
    ws.pw.Tn = c.take<double>((size_t)B * B);
    ws.pw.oz_cap = ozaki::bytes(J, B, B, 1);
    ws.pw.oz = c.take<char>(ws.pw.oz_cap);
    ws.weB = c.take<int>((size_t)B);
    ws.wblobz = c.take<__nv_bfloat16>(ozaki::packed_bytes(B, J, ozaki::kTileB) / 2);
  }
  ws.status = c.take<int>(1);  // last piece: the short forms read it at bytes - 256
  ws.bytes = c.off;
  return ws;
}

// Buffers of the split-precision engine for one stream: packed B operand, packed rank-k
// operands, split-K partial products.
struct SplitBufs {
  __nv_bfloat16 *bblob, *ablob, *rblob;
  double* P;
  size_t P_cap;
};

struct Ge2gbWs {
  double *Yu[2], *Wu[2], *Yv[2], *Wv[2], *Z[2], *ZT, *MT, *P, *splitk[2], *part, *rowbuf, *gram;
  double *ZT2, *P2;  // ge2bb: the panel stream's one-sided products (Variant V1)
  PanelW pw;
  int* sh;           // ge2bb: exponent balance of the two-sided update's operands
  GridSync* gs;
  SplitBufs sb[2];  // [0] caller's stream, [1] panel stream (look-ahead)
  char *ozp[2], *ozr[2];  // Ozaki-scheme buffers per stream (see Sy2sbWs)
  size_t ozp_cap;
  int* status;
  int64_t ldu, ldv;
  size_t splitk_cap;
  size_t bytes;
};

static Ge2gbWs carve_ge2gb(void* work, int64_t m, int64_t n, int64_t w, const Options& o, int sms,
                           bool bb = false) {
  Carver c{static_cast<char*>(work)};
  Ge2gbWs ws{};
  const int64_t b = o.b;
  const int nbuf = o.lookahead == 0 ? 1 : 2;
  ws.ldu = std::max<int64_t>(m, 1);
  ws.ldv = std::max<int64_t>(n, 1);
  for (int q = 0; q < 2; ++q) {
    ws.Yu[q] = q < nbuf ? c.take<double>(ws.ldu * b) : ws.Yu[0];
    ws.Wu[q] = q < nbuf ? c.take<double>(ws.ldu * b) : ws.Wu[0];
  }
  // row-panel Y/W: two pairs with the second look-ahead overlap (w >= 3b), which keeps the
  // previous row panel's reflectors while the next one is factored
  const int nbv = (o.lookahead != 0 && (bb || 3 * b <= w)) ? 2 : 1;
  for (int q = 0; q < 2; ++q) {
    ws.Yv[q] = q < nbv ? c.take<double>(ws.ldv * b) : ws.Yv[0];
    ws.Wv[q] = q < nbv ? c.take<double>(ws.ldv * b) : ws.Wv[0];
  }
  ws.MT = c.take<double>((size_t)b * b);
  ws.ZT = c.take<double>(ws.ldv * b);
  ws.P = c.take<double>(ws.ldu * b);
  if (bb) {
    ws.ZT2 = o.lookahead != 0 ? c.take<double>(ws.ldv * b) : ws.ZT;
    ws.P2 = o.lookahead != 0 ? c.take<double>(ws.ldu * b) : ws.P;
    ws.sh = c.take<int>(2);
  }
  ws.splitk_cap = (size_t)kSmallSplits * b * b * 4;
  for (int q = 0; q < 2; ++q) {
    ws.Z[q] = q < nbuf ? c.take<double>(b * ws.ldv) : ws.Z[0];
    ws.splitk[q] = q < nbuf ? c.take<double>(ws.splitk_cap) : ws.splitk[0];
  }
  ws.rowbuf = c.take<double>(8 * (size_t)b);  // up to four rows per step, two steps
  ws.gram = c.take<double>((size_t)b * b);    // Gram coefficients of the panel (W formed after it)
  ws.gs = c.take<GridSync>(1);  // 256 bytes, immediately followed by the accumulators
  ws.part = c.take<double>((panel_sync_bytes((int)b) - 256) / sizeof(double));
  if (is_split(o)) {
    const int S = split::slices_of(o.precision);
    const int BN = split::stream_bn((int)b);
    const int Kr = (int)((b + 63) / 64 * 64);
    const int64_t big = std::max(ws.ldu, ws.ldv);
    for (int q = 0; q < nbuf; ++q) {
      SplitBufs& sb = ws.sb[q];
      sb.bblob = c.take<__nv_bfloat16>(split::packed_bytes(BN, (int)big, BN, 32, S) / 2);
      sb.ablob = c.take<__nv_bfloat16>(split::packed_bytes((int)big, Kr, 128, 64, S) / 2);
      sb.rblob = c.take<__nv_bfloat16>(split::packed_bytes((int)big, Kr, 128, 64, S) / 2);
      sb.P_cap = (size_t)kMaxStreamSplits * big * BN;
      sb.P = c.take<double>(sb.P_cap);
    }
    if (nbuf == 1) ws.sb[1] = ws.sb[0];
  }
  if (o.precision == BANDRED_OZAKI) {
    const int big = (int)std::max(ws.ldu, ws.ldv), B = (int)b;
    ws.ozp_cap = ozaki::bytes(big, B, big, ozaki::choose_splits(big, B, big, sms));
    ws.pw.Tn = c.take<double>((size_t)B * B);
    ws.pw.oz_cap = ozaki::bytes(big, B, B, 1);
    ws.pw.oz = c.take<char>(ws.pw.oz_cap);
    for (int q = 0; q < nbuf; ++q) {
      ws.ozp[q] = c.take<char>(ws.ozp_cap);
      ws.ozr[q] = c.take<char>(ozaki::bytes(big, big, bb ? 2 * B : B, 1, false));  // ge2bb: rank br + bl
    }
    if (nbuf == 1) {
      ws.ozp[1] = ws.ozp[0];
      ws.ozr[1] = ws.ozr[0];
    }
  }
  ws.status = c.take<int>(1);  // last piece: the short forms read it at bytes - 256
  ws.bytes = c.off;
  return ws;
}

static int current_sms() {
  int dev = 0;
  cudaGetDevice(&dev);
  return device_info(dev).sms;
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call);    \
  } while (0)

// One panel factorisation: QR of the j x bk panel at `A` (rs = 1, cs = lda) or LQ of the
// bk x j row panel (rs = lda, cs = 1).
// W = -Y T of a panel factored in Gram mode: with the Ozaki precision Tn = -T (one small
// kernel) and the product W = Y Tn on the tensor cores; otherwise the FP64 row-parallel
// forward substitution.
static int form_w(int j, int bk, const double* Y, double* W, int64_t ldy, const double* tau, const double* gram,
                  const PanelW* pw, int* status, const Options& o, cudaStream_t s) {
  if (pw && pw->Tn && o.precision == BANDRED_OZAKI) {
    CK(launch_t_from_gram(bk, tau, gram, pw->Tn, s));
    using ozaki::Operand;
    const Operand a{Y, ldy, 0, bk, nullptr, 0, 0, 0, j}, t{pw->Tn, bk, 1, bk, nullptr, 0, 0, 0, bk};
    const int sp = ozaki::fit_splits(j, bk, bk, 1, pw->oz_cap);
    CK(ozaki::product(a, t, j, bk, bk, 1.0, 0.0, W, ldy, ozaki::carve(pw->oz, j, bk, bk, sp), sp, status, o.limit_ns,
                      s));
    return 0;
  }
  CK(launch_w_from_gram(j, bk, Y, tau, gram, W, ldy, s));
  return 0;
}

static int run_panel(double* A, int64_t rs, int64_t cs, int j, int bk, double* tau, double* Y, double* W,
                     int64_t ldy, double* acc, double* rowbuf, double* gram, GridSync* gs, int* status,
                     const Options& o, int max_ctas, unsigned int extra, cudaStream_t s,
                     const PanelW* pw = nullptr) {
  PanelParams p{};
  p.trace = prof::trace_take();
  // Short panels: one thread-block cluster (no grid-wide barrier, deterministic sums).
  // (The phase trace is taken only by the grid panel below.)
  if (cluster_panels(o) && extra == 0) {
    int C = 1;
    while (C < kClusterMax && (j + C - 1) / C > kClusterMinRows) C *= 2;
    const int Rc = (j + C - 1) / C;
    if (Rc <= kClusterRows) {
      p.A = A;
      p.rs = rs;
      p.cs = cs;
      p.j = j;
      p.bk = bk;
      p.R = Rc;
      p.Rp = Rc | 1;
      p.tau = tau;
      p.Y = Y;
      p.W = W;
      p.ldy = ldy;
      p.status = status;
      p.limit_ns = o.limit_ns;
      p.w_in_smem = true;
      p.w_fp32 = is_split(o);
      if (!is_split(o) && bk <= 128) {  // FP64 W formed after the panel, as for the grid panel
        p.G = gram;
        CK(launch_panel_cluster(&p, nullptr, 1, C, p.Rp, bk, s));
        return form_w(j, bk, Y, W, ldy, tau, gram, pw, status, o, s);
      }
      CK(launch_panel_cluster(&p, nullptr, 1, C, p.Rp, bk, s));
      return 0;
    }
  }
  int G, R, Rp;
  bool w_smem = false;
  if (panel_geometry(j, bk, max_ctas, kMinPanelRows, &G, &R, &Rp, &w_smem) != 0) return BANDRED_ERR_UNSUPPORTED;
  p.A = A;
  p.rs = rs;
  p.cs = cs;
  p.j = j;
  p.bk = bk;
  p.R = R;
  p.Rp = Rp;
  p.tau = tau;
  p.Y = Y;
  p.W = W;
  p.ldy = ldy;
  p.acc = acc;
  p.rowbuf = rowbuf;
  p.gs = gs;
  p.status = status;
  p.limit_ns = o.limit_ns;
  p.extra = extra;
  p.w_in_smem = w_smem;
  p.w_fp32 = is_split(o);
  p.phases = prof::phase_take(&p.phase_steps);
  // four reflectors per grid-wide reduction when the caller asks for them and their larger
  // shared-memory footprint fits; pairs otherwise (the default: on GB300 the four-reflector
  // derivation's serial FP64 work costs more than the grid barrier it saves)
  constexpr size_t kSmemMax = 226 * 1024;  // the opt-in limit less the kernel's static shared memory
  if (o.panel_group == 4 && panel4_smem_bytes(bk, Rp, false) <= kSmemMax) {
    p.w_in_smem = panel4_smem_bytes(bk, Rp, true) <= kSmemMax;
    CK(launch_panel4(p, G, s));
    return 0;
  }
  // FP64 W (every precision but the split ones, whose W is FP32 and cheap in the panel): the
  // panel stores its Gram coefficients and a row-parallel kernel forms W after it, keeping
  // that FP64 work off the panel's per-reflector critical path.
  if (!is_split(o) && bk <= 128) {
    p.G = gram;
    p.w_in_smem = false;
    CK(launch_panel(p, G, s));
    return form_w(j, bk, Y, W, ldy, tau, gram, pw, status, o, s);
  }
  CK(launch_panel(p, G, s));
  return 0;
}

// ---------------------------------------------------------------------------------
// Auxiliary stream (highest priority) and events used for look-ahead, one set per host
// thread and device, created by the first look-ahead call of that thread on that device
// and kept (never destroyed) for the thread's later calls.
struct AuxStreams {
  cudaStream_t panel = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

static int aux_streams(AuxStreams** out) {
  thread_local AuxStreams per_dev[kMaxDevices];
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return record_cuda_error(cudaErrorInvalidDevice, "look-ahead streams");
  AuxStreams& a = per_dev[dev];
  if (!a.panel) {
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&a.panel, cudaStreamNonBlocking, hi));
    for (auto& e : a.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  *out = &a;
  return 0;
}

// Split of the streamed product over the reduction dimension: enough CTAs for whole
// waves on `sms` SMs (one CTA per SM), at least two stages per split.
static int stream_splits(int tiles, int nkb, int sms, int cap) {
  int best = 1;
  double best_eff = 0.0;
  for (int sp = 1; sp <= cap; ++sp) {
    if (sp > 1 && nkb / sp < 2) break;
    const int ctas = tiles * sp;
    const int waves = (ctas + sms - 1) / sms;
    const double eff = (double)ctas / ((double)waves * sms);
    if (eff > best_eff + 0.02) {
      best_eff = eff;
      best = sp;
    }
    if (eff >= 0.9) break;
  }
  return best;
}

// SMs for the look-ahead panel of V2 (jp x bp rows and columns) while the rank-2k update of
// the rest of A2 (order j, rank 2 bu) holds the others.  A model of the two durations on
// GB300, fitted (least squares) to device traces of the Ozaki path at n = 8192, w = b = 64:
//   panel  ~ 6.4 us per pair of reflectors (latency) + 5.1e-4 us x jp bp^2 / P,
//   update ~ 1.26e-5 us x j^2 bu / (sms - P),
// and P minimises the larger of the two.  P never drops below the CTA count at which the
// panel's rows still fit in shared memory; fixed > 0 overrides the model.
static int lookahead_panel_ctas(int jp, int bp, int j, int bu, int sms, int fixed, bool cluster) {
  if (cluster && jp <= kClusterMax * kClusterRows) return std::min(kClusterMax, sms - 1);  // a cluster panel
  const int pmax = std::min(sms - 1, (jp + kMinPanelRows - 1) / kMinPanelRows);  // CTAs a grid panel uses
  int pmin = 1;
  while (pmin < sms) {
    int G, Rr, Rp;
    bool wsm;
    if (panel_geometry(jp, bp, pmin, kMinPanelRows, &G, &Rr, &Rp, &wsm) == 0) break;
    ++pmin;
  }
  if (pmin >= sms) return sms;  // only the whole GPU holds the panel: the update waits
  if (fixed > 0) return std::max(pmin, std::min(fixed, sms - 1));
  int best = std::min(pmin, pmax);
  double best_t = 1e300;
  for (int P = pmin; P <= pmax; ++P) {
    const double tp = 6.4 * (bp / 2.0) + 5.1e-4 * (double)jp * bp * bp / P;
    const double tu = 1.26e-5 * (double)j * j * bu / (sms - P);
    const double t = std::max(tp, tu);
    if (t < best_t) {
      best_t = t;
      best = P;
    }
  }
  return best;
}

namespace {

// One sy2sb reduction: the state shared by the steps of an iteration.
struct Sy2sb {
  int64_t n, w, lda;
  double* A;
  double* tau;
  Options o;
  Sy2sbWs ws;
  int* status;
  int sms, pmax, S;
  unsigned int extra;

  // ctas > 0: at most that many CTAs for a grid panel (the look-ahead panel that shares
  // the GPU with the rest of the trailing update)
  int panel(int64_t k, int buf, cudaStream_t s, int ctas = 0) {
    const int bk = (int)std::min<int64_t>(o.b, n - w - 1 - k);
    const int64_t r0 = k + w;
    const int j = (int)(n - r0);
    prof::Scope sc(prof::kPanel, s, panel_flops(j, bk), panel_bytes(j, bk));
    prof::TraceScope tr(prof::kTracePanel, k);
    int rc = run_panel(A + r0 + k * lda, 1, lda, j, bk, tau + k, ws.Y[buf], ws.W[buf], ws.ld, ws.part, ws.rowbuf,
                       ws.gram, ws.gs, status, o, ctas > 0 ? std::min(ctas, pmax) : pmax, extra, s, &ws.pw);
    extra = 0;
    return rc;
  }

  // A1 = A(r0:n, k+bk : k+w) columns [c0, c1) (relative to A1) += Y (W^T A1).
  int update_a1(int64_t k, int buf, int c0, int c1, int zi, cudaStream_t s) {
    const int bk = (int)std::min<int64_t>(o.b, n - w - 1 - k);
    const int64_t r0 = k + w;
    const int j = (int)(n - r0);
    if (c1 <= c0) return 0;
    const int na = c1 - c0;
    double* A1 = A + r0 + (k + bk + c0) * lda;
    const int sp = choose_splits(bk, na, j, ws.splitk_cap, sms);
    prof::Scope sc(prof::kGemm, s, 4.0 * j * na * bk, 8.0 * (2.0 * j * na + 2.0 * j * bk));
    CK(gemm_f64(bk, na, j, 1.0, MatView{ws.W[buf], ws.ld, 1}, MatView{A1, 1, lda}, 0.0, ws.Z[zi], bk, sp,
                ws.splitk[zi], s));
    CK(gemm_f64(j, na, bk, 1.0, MatView{ws.Y[buf], 1, ws.ld}, MatView{ws.Z[zi], 1, bk}, 1.0, A1, lda, 1, nullptr, s));
    return 0;
  }

  // Ozaki buffers of the rank-2k operands [X3 | Y] and [Y | X3] (j rows, K = 2 bk): one
  // row-exponent array serves both, and the second one's space holds the two largest
  // exponents that balance the halves.
  ozaki::Bufs rank2k_bufs(int j, int bk) const {
    ozaki::Bufs b = ozaki::carve(ws.ozr, j, j, 2 * bk, 1);
    b.eB = b.eA;
    return b;
  }
  int* rank2k_shift(int j, int bk) const { return ozaki::carve(ws.ozr, j, j, 2 * bk, 1).eB; }

  // X1 = A2 W, X2 = X1^T W / 2, X3 = X1 + Y X2 (into ws.X); for the split path also packs
  // the operands of the rank-2k update.
  int compute_x(int64_t k, int buf, cudaStream_t s) {
    const int bk = (int)std::min<int64_t>(o.b, n - w - 1 - k);
    const int64_t r0 = k + w;
    const int j = (int)(n - r0);
    const int64_t ld = ws.ld;
    double* A2 = A + r0 + r0 * lda;
    const double* Y = ws.Y[buf];
    const double* W = ws.W[buf];
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const int B = bk;
      const unsigned long long lim = o.limit_ns;
      {
        // X1 = A2 W (A2 symmetric, lower stored; row (n, k) of the right operand is W(k, n))
        prof::Scope sc(prof::kSymm, s, symm_flops(j, bk), symm_bytes(j, bk));
        prof::TraceScope tr(prof::kTraceSymm, k);
        // W's exponents and digits go to their own buffers, which X2 reads again
        const int sp = ozaki::fit_splits(j, B, j, ozaki::choose_splits(j, B, j, sms), ws.ozp_cap);
        const Operand a{A2, lda, 2, j, nullptr, 0, 0, 0, j}, w{W, ld, 1, j, nullptr, 0, 0, 0, B};
        ozaki::Bufs bx = ozaki::carve(ws.ozp, j, B, j, sp);
        bx.eB = ws.weB;
        bx.Bblob = ws.wblobz;
        CK(ozaki::product(a, w, j, B, j, 1.0, 0.0, ws.X, ld, bx, sp, status, lim, s));
      }
      prof::Scope sc(prof::kGemm, s, 4.0 * j * bk * bk, 8.0 * 4.0 * j * bk);
      {
        // X2 = X1^T W / 2, W packed by the X1 product
        const int sp = ozaki::fit_splits(B, B, j, ozaki::choose_splits(B, B, j, sms), ws.ozp_cap);
        const Operand x{ws.X, ld, 1, j, nullptr, 0, 0, 0, B}, w{W, ld, 1, j, nullptr, 0, 0, 0, B};
        ozaki::Bufs bx = ozaki::carve(ws.ozp, B, B, j, sp);
        bx.eB = ws.weB;
        bx.Bblob = ws.wblobz;
        bx.b_packed = true;
        CK(ozaki::product(x, w, B, B, j, 0.5, 0.0, ws.X2, B, bx, sp, status, lim, s));
      }
      {
        // X3 = X1 + Y X2
        const int sp = ozaki::fit_splits(j, B, B, ozaki::choose_splits(j, B, B, sms), ws.ozp_cap);
        const Operand y{Y, ld, 0, B, nullptr, 0, 0, 0, j}, x2{ws.X2, B, 1, B, nullptr, 0, 0, 0, B};
        CK(ozaki::product(y, x2, j, B, B, 1.0, 1.0, ws.X, ld, ozaki::carve(ws.ozp, j, B, B, sp), sp, status, lim, s));
      }
      // operands of A2 += X3 Y^T + Y X3^T: [X3 2^-sigma | Y 2^sigma] and [Y 2^sigma | X3 2^-sigma],
      // whose rows hold the same entries and so share their row exponents; sigma, half the
      // gap between the largest exponents of X3 and Y, keeps Y's digits from falling below
      // the scale of rows dominated by X3 (X3 carries the matrix's magnitude, |Y| <= 1)
      int* sh = rank2k_shift(j, B);
      Operand l{ws.X, ld, 0, B, Y, ld, 0, B, j}, r{Y, ld, 0, B, ws.X, ld, 0, B, j};
      l.sh = r.sh = sh;
      l.shsign = 1;
      r.shsign = -1;
      CK(ozaki::balance(l, sh, s));
      CK(ozaki::prepare(l, r, rank2k_bufs(j, B), s));
      return 0;
    }
    if (!is_split(o)) {
      {
        prof::Scope sc(prof::kSymm, s, symm_flops(j, bk), symm_bytes(j, bk));
        CK(symm_lower_f64(j, bk, A2, lda, W, ld, ws.X, ld, s));
      }
      prof::Scope sc(prof::kGemm, s, 4.0 * j * bk * bk, 8.0 * 4.0 * j * bk);
      const int sp = choose_splits(bk, bk, j, ws.splitk_cap, sms);
      CK(gemm_f64(bk, bk, j, 0.5, MatView{ws.X, ld, 1}, MatView{W, 1, ld}, 0.0, ws.X2, bk, sp, ws.splitk[0], s));
      CK(gemm_f64(j, bk, bk, 1.0, MatView{Y, 1, ld}, MatView{ws.X2, 1, bk}, 1.0, ws.X, ld, 1, nullptr, s));
      return 0;
    }
    const int BN = split::stream_bn(bk);
    const int nkb = (j + 31) / 32;
    {
      prof::Scope sc(prof::kConvert, s, 0.0, 8.0 * j * bk + 2.0 * S * j * BN);
      split::PackParams pp{};
      pp.M1 = W;
      pp.ld1 = ld;
      pp.K1 = j;
      pp.t1 = 1;
      pp.scale1 = pp.scale2 = 1.0;
      pp.R = bk;
      pp.TR = BN;
      pp.TK = 32;
      pp.nrb = 1;
      pp.nkb = nkb;
      pp.S = S;
      pp.out = ws.wblob;
      pp.status = status;
      CK(split::pack(pp, s));
    }
    split::StreamParams sp{};
    sp.Bblob = ws.wblob;
    sp.nkb = nkb;
    sp.N = bk;
    sp.status = status;
    sp.limit_ns = o.limit_ns;
    {
      // X1 = A2 W, A2 symmetric with its lower triangle stored
      prof::Scope sc(prof::kSymm, s, symm_flops(j, bk), symm_bytes(j, bk));
      const int tiles = (j + 127) / 128;
      int splits = stream_splits(tiles, nkb, sms, kMaxStreamSplits);
      sp.A = A2;
      sp.lda = lda;
      sp.mode = split::kModeSymLower;
      sp.M = j;
      sp.K = j;
      sp.stages_per_split = (nkb + splits - 1) / splits;
      splits = (nkb + sp.stages_per_split - 1) / sp.stages_per_split;
      sp.P = ws.P;
      sp.ldp = j;
      sp.split_stride = (int64_t)j * bk;
      CK(split::stream_gemm(sp, S, splits, s));
      CK(split::reduce(j, bk, splits, ws.P, j, (int64_t)j * bk, 1.0, 0.0, ws.X, ld, s));
    }
    prof::Scope sc(prof::kGemm, s, 4.0 * j * bk * bk, 8.0 * 4.0 * j * bk);
    {
      // X2 = X1^T W / 2
      int splits = std::min(kMaxSmallSplits, std::max(1, std::min(sms, nkb / 2)));
      sp.A = ws.X;
      sp.lda = ld;
      sp.mode = split::kModeTrans;
      sp.M = bk;
      sp.K = j;
      sp.stages_per_split = (nkb + splits - 1) / splits;
      splits = (nkb + sp.stages_per_split - 1) / sp.stages_per_split;
      sp.P = ws.P;
      sp.ldp = bk;
      sp.split_stride = (int64_t)bk * bk;
      CK(split::stream_gemm(sp, S, splits, s));
      CK(split::reduce(bk, bk, splits, ws.P, bk, (int64_t)bk * bk, 0.5, 0.0, ws.X2, bk, s));
    }
    {
      // X3 = X1 + Y X2
      split::PackParams pp{};
      pp.M1 = ws.X2;
      pp.ld1 = bk;
      pp.K1 = bk;
      pp.t1 = 1;
      pp.scale1 = pp.scale2 = 1.0;
      pp.R = bk;
      pp.TR = BN;
      pp.TK = 32;
      pp.nrb = 1;
      pp.nkb = (bk + 31) / 32;
      pp.S = S;
      pp.out = ws.x2blob;
      pp.status = status;
      CK(split::pack(pp, s));
      split::StreamParams s3 = sp;
      s3.A = Y;
      s3.lda = ld;
      s3.mode = split::kModePlain;
      s3.M = j;
      s3.K = bk;
      s3.Bblob = ws.x2blob;
      s3.nkb = pp.nkb;
      s3.stages_per_split = pp.nkb;
      s3.P = ws.P;
      s3.ldp = j;
      s3.split_stride = (int64_t)j * bk;
      CK(split::stream_gemm(s3, S, 1, s));
      CK(split::reduce(j, bk, 1, ws.P, j, (int64_t)j * bk, 1.0, 1.0, ws.X, ld, s));
    }
    {
      // operands of A2 += X3 Y^T + Y X3^T: [X3 | Y] and [Y | X3]
      const int Kr = (2 * bk + 63) / 64 * 64;
      split::PackParams pp{};
      pp.M1 = ws.X;
      pp.ld1 = ld;
      pp.K1 = bk;
      pp.t1 = 0;
      pp.M2 = Y;
      pp.ld2 = ld;
      pp.K2 = bk;
      pp.t2 = 0;
      pp.scale1 = pp.scale2 = 1.0;
      pp.R = j;
      pp.TR = 128;
      pp.TK = 64;
      pp.nrb = (j + 127) / 128;
      pp.nkb = Kr / 64;
      pp.S = S;
      pp.out = ws.ablob;
      pp.status = status;
      CK(split::pack(pp, s));
      pp.M1 = Y;
      pp.M2 = ws.X;
      pp.out = ws.bblob;
      CK(split::pack(pp, s));
    }
    return 0;
  }

  // A2 += X3 Y^T + Y X3^T on the lower triangle of A2's columns [c0, c1); max_ctas > 0
  // keeps the update to that many CTAs (Ozaki precision), leaving SMs to the panel.
  int syr2k(int64_t k, int buf, int c0, int c1, cudaStream_t s, int max_ctas = 0) {
    const int bk = (int)std::min<int64_t>(o.b, n - w - 1 - k);
    const int64_t r0 = k + w;
    const int j = (int)(n - r0);
    c1 = std::min(c1, j);
    if (c1 <= c0) return 0;
    double* A2 = A + r0 + r0 * lda;
    prof::Scope sc(prof::kSyr2k, s, syr2k_flops(j, c0, c1, bk), syr2k_bytes(j, c0, c1, bk));
    if (o.precision == BANDRED_OZAKI) {
      prof::TraceScope tr(c0 == 0 && c1 < j ? prof::kTraceRankL : prof::kTraceRankR, k);
      CK(ozaki::rank_apply(j, j, 2 * bk, 1.0, A2, lda, c0, c1, 1, rank2k_bufs(j, bk), status,
                           o.limit_ns, s, max_ctas));
      return 0;
    }
    if (!is_split(o)) {
      CK(syr2k_lower_f64(j, bk, A2, lda, ws.X, ws.ld, ws.Y[buf], ws.ld, c0, c1, s));
      return 0;
    }
    split::RankParams rp{};
    rp.Ablob = ws.ablob;
    rp.Bblob = ws.bblob;
    rp.Kr = (2 * bk + 63) / 64 * 64;
    rp.C = A2;
    rp.ldc = lda;
    rp.M = j;
    rp.N = j;
    rp.col0 = c0;
    rp.col1 = c1;
    rp.lower = 1;
    rp.tj0 = c0 / 128;
    rp.alpha = 1.0;
    rp.status = status;
    rp.limit_ns = o.limit_ns;
    const int ti = (j + 127) / 128;
    const int tj = (c1 - 1) / 128 - rp.tj0 + 1;
    CK(split::rank_update(rp, S, ti, tj, s));
    return 0;
  }
};

}  // namespace

// ---------------------------------------------------------------------------------
// sy2sb: Section 2.1 loop.  Iteration k: panel A0 = A(k+w:n, k:k+bk) (Eq. updateA0),
// A1 = A(k+w:n, k+bk:k+w) := A1 + Y (W^T A1) (Eq. updateA1), and the two-sided update of
// A2 = A(k+w:n, k+w:n) through X1 = A2 W, X2 = X1^T W / 2, X3 = X1 + Y X2,
// A2 += X3 Y^T + Y X3^T (Eqs. updateA2symm .. updateA2syr2k).
//
// Look-ahead (Section 2.2) with two streams: the caller's stream `s` and a highest-
// priority panel stream.  V2 (2b > w): after X3, the panel stream updates the columns of
// A2 that hold the next panel (A2^L) and factors it while `s` updates A2^R.  V1 (2b <= w):
// the next panel lies in A1; the panel stream updates A1^L and factors it while `s`
// updates A1^R and A2.
int sy2sb_run(int64_t n, int64_t w, double* A, int64_t lda, double* tau, const Options& o, void* work,
              int* dev_status, cudaStream_t s) {
  Sy2sb R{};
  R.n = n;
  R.w = w;
  R.A = A;
  R.lda = lda;
  R.tau = tau;
  R.o = o;
  R.sms = current_sms();
  R.ws = carve_sy2sb(work, n, w, o, R.sms);
  R.status = dev_status ? dev_status : R.ws.status;
  R.pmax = panel_max_ctas(R.sms, o);
  R.S = is_split(o) ? split::slices_of(o.precision) : 0;
  R.extra = o.debug ? 1u : 0u;
  CK(cudaMemsetAsync(R.status, 0, sizeof(int), s));
  const int64_t nref = n - w;
  if (nref <= 0) return 0;
  CK(cudaMemsetAsync(tau, 0, sizeof(double) * nref, s));
  const int b = o.b;
  const int la = sy2sb_variant(o, w);
  const int64_t last = n - w - 2;  // panels start at k <= n-w-2

  if (la == 0) {
    int buf = 0;
    for (int64_t k = 0; k <= last; k += b) {
      const int bk = (int)std::min<int64_t>(b, n - w - 1 - k);
      int rc = R.panel(k, buf, s);
      if (rc) return rc;
      if ((rc = R.update_a1(k, buf, 0, (int)(w - bk), 0, s))) return rc;
      if ((rc = R.compute_x(k, buf, s))) return rc;
      if ((rc = R.syr2k(k, buf, 0, (int)(n - k - w), s))) return rc;
    }
    return 0;
  }

  if (last < 0) return 0;  // no panel: every reflector has length <= 1
  // V2's two streams at once: the next panel on P SMs while the rest of the rank-2k update
  // holds the others (the Ozaki update can be held to a CTA count; the other precisions'
  // updates take every SM, so their panel waits for free SMs instead).  P is chosen per
  // iteration (la_split), or fixed by opts->panel_ctas.
  const bool la_split = la == 2 && o.precision == BANDRED_OZAKI;
  AuxStreams* ax = nullptr;
  if (int rc = aux_streams(&ax)) return rc;
  cudaStream_t sp = ax->panel;
  cudaEvent_t ev_fork = ax->ev[0], ev_panel = ax->ev[1];
  // The panel stream starts after everything already queued on s.
  CK(cudaEventRecord(ev_fork, s));
  CK(cudaStreamWaitEvent(sp, ev_fork, 0));
  int rc = R.panel(0, 0, sp);
  if (rc) return rc;
  CK(cudaEventRecord(ev_panel, sp));

  if (sy2sb_depth(o, w) == 2) {
    // Depth 2 (V1 with 3b <= w): when iteration t starts, panels t and t + 1 are factored.
    // The panel stream applies Q_t^T and Q_{t+1}^T to the columns of panel t + 2 (they lie
    // in A1 of both iterations, so no two-sided update reaches them) and factors it while
    // the caller's stream updates the rest of A1 and A2 for iteration t.  Y/W of panels t,
    // t + 1, t + 2 live in buffers t mod 3 ..; evp[t & 1] marks panel t factored.
    cudaEvent_t evp[2] = {ev_panel, ax->ev[2]};
    if (b <= last) {
      const int b1 = (int)std::min<int64_t>(b, n - w - 1 - b);
      if ((rc = R.update_a1(0, 0, 0, b1, 1, sp))) return rc;
      if ((rc = R.panel(b, 1, sp))) return rc;
      CK(cudaEventRecord(evp[1], sp));
    }
    for (int64_t k = 0, t = 0; k <= last; k += b, ++t) {
      const int bt = (int)std::min<int64_t>(b, n - w - 1 - k);
      const int64_t k1 = k + b, k2 = k + 2 * b;
      const int b1 = k1 <= last ? (int)std::min<int64_t>(b, n - w - 1 - k1) : 0;
      const int b2 = k2 <= last ? (int)std::min<int64_t>(b, n - w - 1 - k2) : 0;
      const int bt0 = (int)(t % 3), bt1 = (int)((t + 1) % 3), bt2 = (int)((t + 2) % 3);
      CK(cudaStreamWaitEvent(s, evp[t & 1], 0));  // panel t factored
      if (b2 > 0) {
        CK(cudaEventRecord(ev_fork, s));  // iteration t - 1 done (its A1 update reached panel t + 2)
        CK(cudaStreamWaitEvent(sp, ev_fork, 0));
        if ((rc = R.update_a1(k, bt0, b1, b1 + b2, 1, sp))) return rc;  // Q_t^T (A1 of iteration t)
        if ((rc = R.update_a1(k1, bt1, 0, b2, 1, sp))) return rc;       // Q_{t+1}^T (A1 of t + 1)
        if ((rc = R.panel(k2, bt2, sp))) return rc;
        CK(cudaEventRecord(evp[t & 1], sp));  // panel t + 2: the same parity as t
      }
      // A1 of iteration t without the columns of panels t + 1 and t + 2, then A2
      if ((rc = R.update_a1(k, bt0, b1 + b2, (int)(w - bt), 0, s))) return rc;
      if ((rc = R.compute_x(k, bt0, s))) return rc;
      if ((rc = R.syr2k(k, bt0, 0, (int)(n - k - w), s))) return rc;
    }
    CK(cudaEventRecord(ev_fork, sp));
    CK(cudaStreamWaitEvent(s, ev_fork, 0));
    return 0;
  }

  int buf = 0;
  for (int64_t k = 0; k <= last; k += b, buf ^= 1) {
    const int bk = (int)std::min<int64_t>(b, n - w - 1 - k);
    const int64_t kn = k + b;  // next panel
    const bool has_next = kn <= last;
    const int bkn = has_next ? (int)std::min<int64_t>(b, n - w - 1 - kn) : 0;
    CK(cudaStreamWaitEvent(s, ev_panel, 0));  // panel k done
    const int j = (int)(n - k - w);
    if (la == 2) {
      // V2: A1 (if any), X1..X3 on s; then A2^L + next panel on sp, A2^R on s.
      if ((rc = R.update_a1(k, buf, 0, (int)(w - bk), 0, s))) return rc;
      if ((rc = R.compute_x(k, buf, s))) return rc;
      const int cL = has_next ? (int)std::max<int64_t>(0, b - w + bkn) : 0;
      if (has_next && cL > 0) {
        CK(cudaEventRecord(ev_fork, s));
        CK(cudaStreamWaitEvent(sp, ev_fork, 0));
        // A2^L runs on the SMs the next panel will hold, so that it does not compete with
        // A2^R for the others
        const int la_panel = la_split ? lookahead_panel_ctas(j - b, bkn, j, bk, R.sms, o.panel_ctas, cluster_panels(o)) : 0;
        if ((rc = R.syr2k(k, buf, 0, cL, sp, la_panel))) return rc;
        if ((rc = R.panel(kn, buf ^ 1, sp, la_panel))) return rc;
        CK(cudaEventRecord(ev_panel, sp));
        if ((rc = R.syr2k(k, buf, cL, j, s, la_split ? R.sms - la_panel : 0))) return rc;
      } else {
        if ((rc = R.syr2k(k, buf, 0, j, s))) return rc;
        if (has_next) {
          if ((rc = R.panel(kn, buf ^ 1, s))) return rc;
          CK(cudaEventRecord(ev_panel, s));
        }
      }
    } else {
      // V1: the next panel lies in A1 columns [0, bkn) (relative to A1).
      if (has_next) {
        CK(cudaEventRecord(ev_fork, s));  // iteration k-1's update is complete on s
        CK(cudaStreamWaitEvent(sp, ev_fork, 0));
        if ((rc = R.update_a1(k, buf, 0, bkn, 1, sp))) return rc;
        if ((rc = R.panel(kn, buf ^ 1, sp))) return rc;
        CK(cudaEventRecord(ev_panel, sp));
      }
      if ((rc = R.update_a1(k, buf, has_next ? bkn : 0, (int)(w - bk), 0, s))) return rc;
      if ((rc = R.compute_x(k, buf, s))) return rc;
      if ((rc = R.syr2k(k, buf, 0, j, s))) return rc;
    }
  }
  // Join: everything issued on the panel stream is ordered before later work on s.
  CK(cudaEventRecord(ev_fork, sp));
  CK(cudaStreamWaitEvent(s, ev_fork, 0));
  return 0;
}

size_t sy2sb_workspace_bytes(int64_t n, int64_t w, const Options& o) {
  return carve_sy2sb(nullptr, n, w, o, current_sms()).bytes;
}

// ---------------------------------------------------------------------------------
// Split-precision building blocks shared by the ge2gb steps.
namespace {

// C (M x N) = alpha op(A) Bm + beta C with op(A) M x K streamed from FP64 (mode plain /
// trans) and Bm the K x N FP64 matrix Bsrc[k + n*ldb] (packed here).
int split_product(int M, int N, int K, const double* A, int64_t lda, int mode, const double* Bsrc, int64_t ldb,
                  double alpha, double beta, double* C, int64_t ldc, const SplitBufs& sb, int S, int sms, int* status,
                  unsigned long long limit_ns, cudaStream_t s) {
  if (M <= 0 || N <= 0) return 0;
  // algorithmic: one read of op(A) and of Bm, one write of C
  prof::Scope sc(prof::kStream, s, 2.0 * M * N * K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
  const int BN = split::stream_bn(N);
  const int nkb = (K + 31) / 32;
  split::PackParams pp{};
  pp.M1 = Bsrc;
  pp.ld1 = ldb;
  pp.K1 = K;
  pp.t1 = 1;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = N;
  pp.TR = BN;
  pp.TK = 32;
  pp.nrb = 1;
  pp.nkb = std::max(nkb, 1);
  pp.S = S;
  pp.out = sb.bblob;
  pp.status = status;
  CK(split::pack(pp, s));
  split::StreamParams sp{};
  sp.A = A;
  sp.lda = lda;
  sp.mode = mode;
  sp.M = M;
  sp.K = K;
  sp.N = N;
  sp.Bblob = sb.bblob;
  sp.nkb = pp.nkb;
  const int tiles = (M + 127) / 128;
  int splits = stream_splits(tiles, pp.nkb, sms, kMaxStreamSplits);
  while (splits > 1 && (size_t)splits * M * N > sb.P_cap) --splits;
  sp.stages_per_split = (pp.nkb + splits - 1) / splits;
  splits = (pp.nkb + sp.stages_per_split - 1) / sp.stages_per_split;
  sp.P = sb.P;
  sp.ldp = M;
  sp.split_stride = (int64_t)M * N;
  sp.status = status;
  sp.limit_ns = limit_ns;
  CK(split::stream_gemm(sp, S, splits, s));
  CK(split::reduce(M, N, splits, sb.P, M, (int64_t)M * N, alpha, beta, C, ldc, s));
  return 0;
}

// C (M x N) += Am Bm^T with Am (M x K) and Bm (N x K) FP64 column-major, K <= 128.
int split_rank(int M, int N, int K, const double* Am, int64_t lda, const double* Bm, int64_t ldb, double* C,
               int64_t ldc, const SplitBufs& sb, int S, int* status, unsigned long long limit_ns, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return 0;
  // algorithmic: C read and written once, Am and Bm read once
  prof::Scope sc(prof::kRank, s, 2.0 * M * N * K, 8.0 * (2.0 * M * N + (double)(M + N) * K));
  const int Kr = (K + 63) / 64 * 64;
  split::PackParams pp{};
  pp.M1 = Am;
  pp.ld1 = lda;
  pp.K1 = K;
  pp.t1 = 0;
  pp.K2 = 0;
  pp.scale1 = pp.scale2 = 1.0;
  pp.R = M;
  pp.TR = 128;
  pp.TK = 64;
  pp.nrb = (M + 127) / 128;
  pp.nkb = Kr / 64;
  pp.S = S;
  pp.out = sb.ablob;
  pp.status = status;
  CK(split::pack(pp, s));
  pp.M1 = Bm;
  pp.ld1 = ldb;
  pp.R = N;
  pp.nrb = (N + 127) / 128;
  pp.out = sb.rblob;
  CK(split::pack(pp, s));
  split::RankParams rp{};
  rp.Ablob = sb.ablob;
  rp.Bblob = sb.rblob;
  rp.Kr = Kr;
  rp.C = C;
  rp.ldc = ldc;
  rp.M = M;
  rp.N = N;
  rp.col0 = 0;
  rp.col1 = N;
  rp.lower = 0;
  rp.tj0 = 0;
  rp.alpha = 1.0;
  rp.status = status;
  rp.limit_ns = limit_ns;
  CK(split::rank_update(rp, S, (M + 127) / 128, (N + 127) / 128, s));
  return 0;
}

struct Ge2gb {
  int64_t m, n, w, lda;
  double* A;
  double *tauq, *taup;
  Options o;
  Ge2gbWs ws;
  int* status;
  int sms, pmax, S;
  unsigned int extra;

  int bk_of(int64_t k) const { return (int)std::min<int64_t>(o.b, n - k); }

  // QR of B = A(k:m, k:k+bk) (Eq. updateB); ctas > 0 caps the panel's CTAs.
  int left_panel(int64_t k, int buf, cudaStream_t s, int ctas = 0) {
    const int bk = bk_of(k);
    const int j = (int)(m - k);
    prof::Scope sc(prof::kPanel, s, panel_flops(j, bk), panel_bytes(j, bk));
    prof::TraceScope tr(prof::kTracePanel, k);
    int rc = run_panel(A + k + k * lda, 1, lda, j, bk, tauq + k, ws.Yu[buf], ws.Wu[buf], ws.ldu, ws.part,
                       ws.rowbuf, ws.gram, ws.gs, status, o, ctas > 0 ? std::min(ctas, pmax) : pmax, extra, s,
                       &ws.pw);
    extra = 0;
    return rc;
  }

  // E = A(k:m, k+bk:n) columns [c0, c1) += Y_U (W_U^T E) (Eq. updateCD).
  int e_update(int64_t k, int buf, int c0, int c1, int q, cudaStream_t s) {
    const int bk = bk_of(k);
    const int j = (int)(m - k);
    c1 = std::min<int>(c1, (int)(n - k - bk));
    if (c1 <= c0) return 0;
    const int nc = c1 - c0;
    double* E = A + k + (k + bk + c0) * lda;
    if (o.precision == BANDRED_FP64) {
      prof::Scope sc(prof::kGemm, s, 4.0 * j * nc * bk, 8.0 * (3.0 * j * nc + 2.0 * j * bk));
      const int sp = choose_splits(bk, nc, j, ws.splitk_cap, sms);
      CK(gemm_f64(bk, nc, j, 1.0, MatView{ws.Wu[buf], ws.ldu, 1}, MatView{E, 1, lda}, 0.0, ws.Z[q], bk, sp,
                  ws.splitk[q], s));
      CK(gemm_f64(j, nc, bk, 1.0, MatView{ws.Yu[buf], 1, ws.ldu}, MatView{ws.Z[q], 1, bk}, 1.0, E, lda, 1, nullptr,
                  s));
      return 0;
    }
    // Z^T = E^T W_U (nc x bk), then E += Y_U (Z^T)^T
    double* ZT = ws.ZT + c0;
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const Operand et{E, lda, 1, j, nullptr, 0, 0, 0, nc}, wu{ws.Wu[buf], ws.ldu, 1, j, nullptr, 0, 0, 0, bk};
      {
        prof::Scope sc(prof::kStream, s, 2.0 * nc * bk * j, 8.0 * ((double)j * nc + (double)j * bk + (double)nc * bk));
        const int sp = ozaki::fit_splits(nc, bk, j, ozaki::choose_splits(nc, bk, j, sms), ws.ozp_cap);
        CK(ozaki::product(et, wu, nc, bk, j, 1.0, 0.0, ZT, ws.ldv, ozaki::carve(ws.ozp[q], nc, bk, j, sp), sp, status,
                          o.limit_ns, s));
      }
      prof::Scope sc(prof::kRank, s, 2.0 * j * nc * bk, 8.0 * (2.0 * j * nc + (double)(j + nc) * bk));
      const Operand yu{ws.Yu[buf], ws.ldu, 0, bk, nullptr, 0, 0, 0, j}, zt{ZT, ws.ldv, 0, bk, nullptr, 0, 0, 0, nc};
      const ozaki::Bufs rb = ozaki::carve(ws.ozr[q], j, nc, bk, 1);
      CK(ozaki::prepare(yu, zt, rb, s));
      prof::TraceScope tr(prof::kTraceLeft, k);
      CK(ozaki::rank_apply(j, nc, bk, 1.0, E, lda, 0, nc, 0, rb, status, o.limit_ns, s));
      return 0;
    }
    if (int rc = split_product(nc, bk, j, E, lda, split::kModeTrans, ws.Wu[buf], ws.ldu, 1.0, 0.0, ZT, ws.ldv,
                               ws.sb[q], S, sms, status, o.limit_ns, s))
      return rc;
    return split_rank(j, nc, bk, ws.Yu[buf], ws.ldu, ZT, ws.ldv, E, lda, ws.sb[q], S, status, o.limit_ns, s);
  }

  // ---- building blocks of the second look-ahead overlap (ge2gb_run, w >= 3b), in the
  // precision of the options; q selects the stream's buffers (0 caller, 1 panel stream).
  // C (M x N, ldc) = As^T Bs with As K x M (lda) and Bs K x N (ldb), column-major.
  int prod_t(int M, int N, int K, const double* As, int64_t lda, const double* Bs, int64_t ldb, double* C, int64_t ldc,
             int q, cudaStream_t s) {
    if (M <= 0 || N <= 0) return 0;
    prof::Scope sc(prof::kStream, s, 2.0 * M * N * K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
    if (o.precision == BANDRED_FP64) {
      const int sp = choose_splits(M, N, K, ws.splitk_cap, sms);
      CK(gemm_f64(M, N, K, 1.0, MatView{As, lda, 1}, MatView{Bs, 1, ldb}, 0.0, C, ldc, sp, ws.splitk[q], s));
      return 0;
    }
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const Operand a{As, lda, 1, K, nullptr, 0, 0, 0, M}, bo{Bs, ldb, 1, K, nullptr, 0, 0, 0, N};
      const int sp = ozaki::fit_splits(M, N, K, ozaki::choose_splits(M, N, K, sms), ws.ozp_cap);
      CK(ozaki::product(a, bo, M, N, K, 1.0, 0.0, C, ldc, ozaki::carve(ws.ozp[q], M, N, K, sp), sp, status, o.limit_ns,
                        s));
      return 0;
    }
    return split_product(M, N, K, As, lda, split::kModeTrans, Bs, ldb, 1.0, 0.0, C, ldc, ws.sb[q], S, sms, status,
                         o.limit_ns, s);
  }
  // C (M x N, ldc) = As Bs with As M x K (lda) and Bs K x N (ldb).
  int prod_n(int M, int N, int K, const double* As, int64_t lda, const double* Bs, int64_t ldb, double* C, int64_t ldc,
             int q, cudaStream_t s) {
    if (M <= 0 || N <= 0) return 0;
    prof::Scope sc(prof::kStream, s, 2.0 * M * N * K, 8.0 * ((double)M * K + (double)K * N + (double)M * N));
    if (o.precision == BANDRED_FP64) {
      const int sp = choose_splits(M, N, K, ws.splitk_cap, sms);
      CK(gemm_f64(M, N, K, 1.0, MatView{As, 1, lda}, MatView{Bs, 1, ldb}, 0.0, C, ldc, sp, ws.splitk[q], s));
      return 0;
    }
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const Operand a{As, lda, 0, K, nullptr, 0, 0, 0, M}, bo{Bs, ldb, 1, K, nullptr, 0, 0, 0, N};
      const int sp = ozaki::fit_splits(M, N, K, ozaki::choose_splits(M, N, K, sms), ws.ozp_cap);
      CK(ozaki::product(a, bo, M, N, K, 1.0, 0.0, C, ldc, ozaki::carve(ws.ozp[q], M, N, K, sp), sp, status, o.limit_ns,
                        s));
      return 0;
    }
    return split_product(M, N, K, As, lda, split::kModePlain, Bs, ldb, 1.0, 0.0, C, ldc, ws.sb[q], S, sms, status,
                         o.limit_ns, s);
  }
  // C (M x N, ldc) += L R^T with L M x K (ldl) and R N x K (ldr); max_ctas > 0 holds the
  // Ozaki update to that many CTAs (SMs left to a panel on the other stream).
  int rank_k(int M, int N, int K, const double* L, int64_t ldl, const double* Rm, int64_t ldr, double* C, int64_t ldc,
             int q, cudaStream_t s, int max_ctas = 0) {
    if (M <= 0 || N <= 0 || K <= 0) return 0;
    prof::Scope sc(prof::kRank, s, 2.0 * M * N * K, 8.0 * (2.0 * M * N + (double)(M + N) * K));
    if (o.precision == BANDRED_FP64) {
      CK(gemm_f64(M, N, K, 1.0, MatView{L, 1, ldl}, MatView{Rm, ldr, 1}, 1.0, C, ldc, 1, nullptr, s));
      return 0;
    }
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const Operand l{L, ldl, 0, K, nullptr, 0, 0, 0, M}, r{Rm, ldr, 0, K, nullptr, 0, 0, 0, N};
      const ozaki::Bufs rb = ozaki::carve(ws.ozr[q], M, N, K, 1);
      CK(ozaki::prepare(l, r, rb, s));
      CK(ozaki::rank_apply(M, N, K, 1.0, C, ldc, 0, N, 0, rb, status, o.limit_ns, s, max_ctas));
      return 0;
    }
    return split_rank(M, N, K, L, ldl, Rm, ldr, C, ldc, ws.sb[q], S, status, o.limit_ns, s);
  }

  // LQ of C = A(k:k+bkr, k+w:n) (Eq. updateC) into row-panel buffer bvi; ctas > 0 caps the
  // panel's CTAs.
  int right_panel(int64_t k, cudaStream_t s, int bvi = 0, int ctas = 0) {
    const int bk = bk_of(k);
    const int64_t bkr = std::min<int64_t>(bk, n - w - 1 - k);
    if (bkr <= 0) return 0;
    const int jr = (int)(n - k - w);
    prof::Scope sc(prof::kPanel, s, panel_flops(jr, (int)bkr), panel_bytes(jr, (int)bkr));
    prof::TraceScope tr(prof::kTracePanelRow, k);
    return run_panel(A + k + (k + w) * lda, lda, 1, jr, (int)bkr, taup + k, ws.Yv[bvi], ws.Wv[bvi], ws.ldv, ws.part,
                     ws.rowbuf, ws.gram, ws.gs, status, o, ctas > 0 ? std::min(ctas, pmax) : pmax, 0u, s, &ws.pw);
  }

  // D = A(k+bkr:m, k+w:n) += (D W_V) Y_V^T (Eq. updateD), row panel from buffer bvi.
  int d_update(int64_t k, cudaStream_t s, int bvi = 0) {
    const double* Yv = ws.Yv[bvi];
    const double* Wv = ws.Wv[bvi];
    const int bk = bk_of(k);
    const int64_t bkr = std::min<int64_t>(bk, n - w - 1 - k);
    if (bkr <= 0) return 0;
    const int jr = (int)(n - k - w);
    const int nrow = (int)(m - k - bkr);
    if (nrow <= 0) return 0;
    double* D = A + (k + bkr) + (k + w) * lda;
    if (o.precision == BANDRED_FP64) {
      prof::Scope sc(prof::kGemm, s, 4.0 * nrow * jr * bkr, 8.0 * (3.0 * nrow * jr + 2.0 * nrow * bkr));
      const int sp = choose_splits(nrow, (int)bkr, jr, ws.splitk_cap, sms);
      CK(gemm_f64(nrow, (int)bkr, jr, 1.0, MatView{D, 1, lda}, MatView{Wv, 1, ws.ldv}, 0.0, ws.P, ws.ldu, sp,
                  ws.splitk[0], s));
      CK(gemm_f64(nrow, jr, (int)bkr, 1.0, MatView{ws.P, 1, ws.ldu}, MatView{Yv, ws.ldv, 1}, 1.0, D, lda, 1,
                  nullptr, s));
      return 0;
    }
    if (o.precision == BANDRED_OZAKI) {
      using ozaki::Operand;
      const int B = (int)bkr;
      const Operand d{D, lda, 0, jr, nullptr, 0, 0, 0, nrow}, wv{Wv, ws.ldv, 1, jr, nullptr, 0, 0, 0, B};
      {
        prof::Scope sc(prof::kStream, s, 2.0 * nrow * B * jr, 8.0 * ((double)nrow * jr + (double)jr * B + (double)nrow * B));
        const int sp = ozaki::fit_splits(nrow, B, jr, ozaki::choose_splits(nrow, B, jr, sms), ws.ozp_cap);
        CK(ozaki::product(d, wv, nrow, B, jr, 1.0, 0.0, ws.P, ws.ldu, ozaki::carve(ws.ozp[0], nrow, B, jr, sp), sp,
                          status, o.limit_ns, s));
      }
      prof::Scope sc(prof::kRank, s, 2.0 * nrow * jr * B, 8.0 * (2.0 * nrow * jr + (double)(nrow + jr) * B));
      const Operand pp{ws.P, ws.ldu, 0, B, nullptr, 0, 0, 0, nrow}, yv{Yv, ws.ldv, 0, B, nullptr, 0, 0, 0, jr};
      const ozaki::Bufs rb = ozaki::carve(ws.ozr[0], nrow, jr, B, 1);
      CK(ozaki::prepare(pp, yv, rb, s));
      prof::TraceScope tr(prof::kTraceRight, k);
      CK(ozaki::rank_apply(nrow, jr, B, 1.0, D, lda, 0, jr, 0, rb, status, o.limit_ns, s));
      return 0;
    }
    if (int rc = split_product(nrow, (int)bkr, jr, D, lda, split::kModePlain, Wv, ws.ldv, 1.0, 0.0, ws.P, ws.ldu,
                               ws.sb[0], S, sms, status, o.limit_ns, s))
      return rc;
    return split_rank(nrow, jr, (int)bkr, ws.P, ws.ldu, Yv, ws.ldv, D, lda, ws.sb[0], S, status, o.limit_ns, s);
  }
};

}  // namespace

// ---------------------------------------------------------------------------------
// ge2gb: Section 3.1 loop.  Iteration k: QR of B = A(k:m, k:k+bk) (Eq. updateB),
// E = A(k:m, k+bk:n) += Y_U (W_U^T E) (Eq. updateCD), LQ of C = A(k:k+bkr, k+w:n)
// (Eq. updateC), D = A(k+bkr:m, k+w:n) += (D W_V) Y_V^T (Eq. updateD).
//
// Look-ahead (Section 3.2): with w >= 2b the next column panel lies in the first b
// columns of E and is untouched by this iteration's right update, so the panel stream
// updates those columns and factors the next panel while the caller's stream finishes
// the left update; the row panel follows on the panel stream (panels never run
// concurrently: they share their reduction scratch), then the right update on the
// caller's stream.  With w >= 3b (and lookahead -1 or 2) both overlaps of the paper's
// third case run, below.  With w < 2b the steps run in order.
int ge2gb_run(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
              const Options& o, void* work, int* dev_status, cudaStream_t s) {
  if (n > m) {
    // m < n: Section 3.1's reduction of the tall A^T (n x m) = U' B' V'^T, written back
    // transposed: A = V' B'^T U'^T with B'^T lower band.  A^T lives at the front of the
    // workspace; the left reflectors of A^T are A's right ones (taup, m of them), its
    // right reflectors A's left ones (tauq, max(m - w, 0)).
    double* T = static_cast<double*>(work);
    void* rest = static_cast<char*>(work) + align_up((size_t)m * n * sizeof(double));
    CK(transpose_f64((int)m, (int)n, A, lda, T, n, s));
    if (int rc = ge2gb_run(n, m, w, T, n, taup, tauq, o, rest, dev_status, s)) return rc;
    CK(transpose_f64((int)n, (int)m, T, n, A, lda, s));
    return 0;
  }
  Ge2gb R{};
  R.m = m;
  R.n = n;
  R.w = w;
  R.A = A;
  R.lda = lda;
  R.tauq = tauq;
  R.taup = taup;
  R.o = o;
  R.sms = current_sms();
  R.ws = carve_ge2gb(work, m, n, w, o, R.sms);
  R.status = dev_status ? dev_status : R.ws.status;
  R.pmax = panel_max_ctas(R.sms, o);
  R.S = is_split(o) ? split::slices_of(o.precision) : 0;
  R.extra = o.debug ? 1u : 0u;
  CK(cudaMemsetAsync(R.status, 0, sizeof(int), s));
  if (n <= 0) return 0;
  CK(cudaMemsetAsync(tauq, 0, sizeof(double) * n, s));
  if (n - w > 0) CK(cudaMemsetAsync(taup, 0, sizeof(double) * (n - w), s));
  const int b = o.b;
  const bool la = o.lookahead != 0 && 2 * b <= w && n > b;
  int rc;
  if (!la) {
    for (int64_t k = 0; k < n; k += b) {
      if ((rc = R.left_panel(k, 0, s))) return rc;
      if ((rc = R.e_update(k, 0, 0, (int)n, 0, s))) return rc;
      if ((rc = R.right_panel(k, s))) return rc;
      if ((rc = R.d_update(k, s))) return rc;
    }
    return 0;
  }
  AuxStreams* ax = nullptr;
  if ((rc = aux_streams(&ax))) return rc;
  cudaStream_t sp = ax->panel;
  cudaEvent_t ev_fork = ax->ev[0], ev_panel = ax->ev[1], ev_e = ax->ev[2];
  CK(cudaEventRecord(ev_fork, s));
  CK(cudaStreamWaitEvent(sp, ev_fork, 0));
  if ((rc = R.left_panel(0, 0, sp))) return rc;
  CK(cudaEventRecord(ev_panel, sp));

  if (3 * b <= w && (o.lookahead == -1 || o.lookahead == 2)) {
    // Both overlaps of Section 3.2's third case (w >= 3b): the row panel L^k V^k runs beside
    // the right update of the previous iteration, and the next column panel beside the left
    // update.  The left update U_k^T (rows >= k) and the pending right update V_{k-1}
    // (columns >= k - b + w) commute, so both are written from products of the state before
    // either: Z = W_U^T E, P = D W_V and Z V = Z + (Z W_V) Y_V^T give
    //   U_k^T A V_{k-1} = A + P Y_V^T + Y_U (Z V)      (on the rows >= k of E and D).
    // The panel stream applies that to row block k (b rows) and factors L^k V^k, then to the
    // next column panel's columns (below the row block) and factors it, while the caller's
    // stream applies it to everything else.  Iterations with a narrower last panel finish
    // without look-ahead.
    int64_t k = 0, kprev = -1;
    int bu = 0, bvp = 0;
    for (; k + 2 * b <= n - w - 1; k += b, bu ^= 1) {
      const int bk = b, j = (int)(m - k), nc = (int)(n - k - bk);
      double* E = A + k + (k + bk) * lda;
      CK(cudaStreamWaitEvent(s, ev_panel, 0));  // column panel k (and row panel kprev) factored
      // pre-state products on the caller's stream: Z^T = E^T W_U (nc x bk)
      if ((rc = R.prod_t(nc, bk, j, E, lda, R.ws.Wu[bu], R.ws.ldu, R.ws.ZT, R.ws.ldv, 0, s))) return rc;
      int c0v = 0, jr = 0;
      if (kprev >= 0) {
        c0v = (int)(kprev + w - (k + bk));  // first column of E in the pending right update's range
        jr = (int)(n - (kprev + w));
        // P = D W_V, D = A(k:m, kprev+w:n) (its rows start at kprev + b = k)
        if ((rc = R.prod_n(j, b, jr, A + k + (kprev + w) * lda, lda, R.ws.Wv[bvp], R.ws.ldv, R.ws.P, R.ws.ldu, 0, s)))
          return rc;
        // Z V on that range: (Z V)^T = Z^T + Y_V MT^T with MT = (Z^T)^T W_V restricted to it
        if ((rc = R.prod_t(bk, b, jr, R.ws.ZT + c0v, R.ws.ldv, R.ws.Wv[bvp], R.ws.ldv, R.ws.MT, bk, 0, s))) return rc;
        if ((rc = R.rank_k(jr, bk, b, R.ws.Yv[bvp], R.ws.ldv, R.ws.MT, bk, R.ws.ZT + c0v, R.ws.ldv, 0, s))) return rc;
      }
      CK(cudaEventRecord(ev_e, s));
      CK(cudaStreamWaitEvent(sp, ev_e, 0));
      const int bkn = R.bk_of(k + b);
      // With the Ozaki precision the panels hold P SMs and the caller's updates the others
      // (the model of the look-ahead split, with the two rank-b updates of j rows as the
      // update), so both streams run at once; other precisions take every SM.
      const int P = o.precision == BANDRED_OZAKI
                        ? lookahead_panel_ctas(std::max(jr, j - bk), b, j, 2 * b, R.sms, o.panel_ctas, cluster_panels(o))
                        : 0;
      const int rest = P > 0 && P < R.sms ? R.sms - P : 0;
      // panel stream: row block k (rows k .. k+bk), then row panel k; the next column
      // panel's columns below the row block, then that panel
      if ((rc = R.rank_k(bk, nc, bk, R.ws.Yu[bu], R.ws.ldu, R.ws.ZT, R.ws.ldv, E, lda, 1, sp))) return rc;
      if (kprev >= 0 &&
          (rc = R.rank_k(bk, jr, b, R.ws.P, R.ws.ldu, R.ws.Yv[bvp], R.ws.ldv, A + k + (kprev + w) * lda, lda, 1, sp)))
        return rc;
      if ((rc = R.right_panel(k, sp, bvp ^ 1, P))) return rc;
      if ((rc = R.rank_k(j - bk, bkn, bk, R.ws.Yu[bu] + bk, R.ws.ldu, R.ws.ZT, R.ws.ldv, E + bk, lda, 1, sp)))
        return rc;
      if ((rc = R.left_panel(k + b, bu ^ 1, sp, P))) return rc;
      CK(cudaEventRecord(ev_panel, sp));
      // caller's stream: the rest (rows below the row block, columns past the next panel);
      // the pending right update first, so that it is the one beside the row panel (the
      // two are additive updates from the same pre-state products and commute)
      if (kprev >= 0) {
        prof::TraceScope tr(prof::kTraceRight, kprev);
        if ((rc = R.rank_k(j - bk, jr, b, R.ws.P + bk, R.ws.ldu, R.ws.Yv[bvp], R.ws.ldv,
                           A + k + bk + (kprev + w) * lda, lda, 0, s, rest)))
          return rc;
      }
      {
        prof::TraceScope tr(prof::kTraceLeft, k);
        if ((rc = R.rank_k(j - bk, nc - bkn, bk, R.ws.Yu[bu] + bk, R.ws.ldu, R.ws.ZT + bkn, R.ws.ldv,
                           E + bk + (int64_t)bkn * lda, lda, 0, s, rest)))
          return rc;
      }
      kprev = k;
      bvp ^= 1;
    }
    // the rest without look-ahead: the pending right update, then iteration k onwards
    // (column panel k is already factored, in buffer bu)
    CK(cudaStreamWaitEvent(s, ev_panel, 0));
    if (kprev >= 0 && (rc = R.d_update(kprev, s, bvp))) return rc;
    for (bool first = true; k < n; k += b, bu ^= 1, first = false) {
      if (!first && (rc = R.left_panel(k, bu, s))) return rc;
      if ((rc = R.e_update(k, bu, 0, (int)n, 0, s))) return rc;
      if ((rc = R.right_panel(k, s, 0))) return rc;
      if ((rc = R.d_update(k, s, 0))) return rc;
    }
    CK(cudaEventRecord(ev_fork, sp));
    CK(cudaStreamWaitEvent(s, ev_fork, 0));
    return 0;
  }

  int buf = 0;
  for (int64_t k = 0; k < n; k += b, buf ^= 1) {
    const int64_t kn = k + b;
    const bool has_next = kn < n;
    CK(cudaStreamWaitEvent(s, ev_panel, 0));  // left panel k done
    if (has_next) {
      const int bkn = R.bk_of(kn);
      CK(cudaEventRecord(ev_fork, s));  // iteration k-1 is complete on s
      CK(cudaStreamWaitEvent(sp, ev_fork, 0));
      if ((rc = R.e_update(k, buf, 0, bkn, 1, sp))) return rc;
      if ((rc = R.left_panel(kn, buf ^ 1, sp))) return rc;
      if ((rc = R.e_update(k, buf, bkn, (int)n, 0, s))) return rc;
      CK(cudaEventRecord(ev_e, s));
      CK(cudaStreamWaitEvent(sp, ev_e, 0));
      if ((rc = R.right_panel(k, sp))) return rc;
      CK(cudaEventRecord(ev_panel, sp));  // covers left panel k+1 and row panel k
      CK(cudaStreamWaitEvent(s, ev_panel, 0));
    } else {
      if ((rc = R.e_update(k, buf, 0, (int)n, 0, s))) return rc;
      if ((rc = R.right_panel(k, s))) return rc;
    }
    if ((rc = R.d_update(k, s))) return rc;
  }
  CK(cudaEventRecord(ev_fork, sp));
  CK(cudaStreamWaitEvent(s, ev_fork, 0));
  return 0;
}

// ---------------------------------------------------------------------------------
// ge2bb: band with lower and upper bandwidth w, Section 3.3 (Eqs. updateB0 .. gebrd_2k).
// Iteration k: QR of the column panel A(k+w:m, k:k+bl) and LQ of the row panel
// A(k:k+br, k+w:n) (independent: the left reflectors act on rows >= k+w, the right ones on
// columns >= k+w); the one-sided updates of B1 = A(k+w:m, k+bl:k+w) and
// C1 = A(k+br:k+w, k+w:n); and D = A(k+w:m, k+w:n) := Q_L^T D Q_R written as one two-sided
// update from products of D: Z_L = D^T W_L, Z_R = D W_R, X = Z_R + Y_L (Z_L^T W_R),
// D += X Y_R^T + Y_L Z_L^T (Eq. gebrd_2k).
//
// Look-ahead (the panels of iteration k + b on a second stream):
//   V1 (2b <= w): the next column panel lies in the first b columns of B1 and the next row
//     panel in the first b rows of C1, which only one-sided updates reach.  The panel stream
//     updates those columns and rows and factors both panels while the caller's stream
//     updates the rest of B1 and C1 and all of D.
//   V2 (2b > w): with t = 2b - w, the next panels lie in B1, C1 and the first t columns and
//     first t rows of D.  After the products of D, the panel stream applies the two-sided
//     update to D(:, 0:t) and D(0:t, t:) and factors both panels, while the caller's
//     stream updates D(t:, t:), the 2 x 2 partition of D.
namespace {

struct Ge2bb {
  Ge2gb R;  // precision-dispatched products and panels of the ge2gb driver
  int64_t m, n, w, nlq, nrq;
  int b;

  int bl_of(int64_t k) const { return (int)std::max<int64_t>(0, std::min<int64_t>(b, nlq - k)); }
  int br_of(int64_t k) const { return (int)std::max<int64_t>(0, std::min<int64_t>(b, nrq - k)); }
  int jl_of(int64_t k) const { return (int)(m - k - w); }
  int jr_of(int64_t k) const { return (int)(n - k - w); }
  bool lq(int64_t k) const { return bl_of(k) > 0 && jl_of(k) >= 2; }
  bool rq(int64_t k) const { return br_of(k) > 0 && jr_of(k) >= 2; }

  // QR of the column panel and LQ of the row panel of iteration k into buffer q; ctas > 0
  // caps their CTAs.
  int panels(int64_t k, int q, cudaStream_t s, int ctas = 0) {
    Ge2gbWs& ws = R.ws;
    const int pm = ctas > 0 ? std::min(ctas, R.pmax) : R.pmax;
    int rc;
    if (lq(k)) {
      const int jl = jl_of(k), bl = bl_of(k);
      prof::Scope sc(prof::kPanel, s, panel_flops(jl, bl), panel_bytes(jl, bl));
      prof::TraceScope tr(prof::kTracePanel, k);
      if ((rc = run_panel(R.A + (k + w) + k * R.lda, 1, R.lda, jl, bl, R.tauq + k, ws.Yu[q], ws.Wu[q], ws.ldu, ws.part,
                          ws.rowbuf, ws.gram, ws.gs, R.status, R.o, pm, 0u, s, &ws.pw)))
        return rc;
    }
    if (rq(k)) {
      const int jr = jr_of(k), br = br_of(k);
      prof::Scope sc(prof::kPanel, s, panel_flops(jr, br), panel_bytes(jr, br));
      prof::TraceScope tr(prof::kTracePanelRow, k);
      if ((rc = run_panel(R.A + k + (k + w) * R.lda, R.lda, 1, jr, br, R.taup + k, ws.Yv[q], ws.Wv[q], ws.ldv, ws.part,
                          ws.rowbuf, ws.gram, ws.gs, R.status, R.o, pm, 0u, s, &ws.pw)))
        return rc;
    }
    return 0;
  }

  // B1 columns [c0, c1) += Y_L (W_L^T B1) (Eq. updateB1), products into Z (ldz = ldv).
  int b1_update(int64_t k, int q, int c0, int c1, double* Z, int qs, cudaStream_t s) {
    if (!lq(k)) return 0;
    const int bl = bl_of(k), jl = jl_of(k);
    c1 = std::min<int>(c1, (int)std::min<int64_t>(w - bl, n - k - bl));
    if (c1 <= c0) return 0;
    double* B1 = R.A + (k + w) + (k + bl + c0) * R.lda;
    int rc;
    if ((rc = R.prod_t(c1 - c0, bl, jl, B1, R.lda, R.ws.Wu[q], R.ws.ldu, Z, R.ws.ldv, qs, s))) return rc;
    return R.rank_k(jl, c1 - c0, bl, R.ws.Yu[q], R.ws.ldu, Z, R.ws.ldv, B1, R.lda, qs, s);
  }

  // C1 rows [r0, r1) += (C1 W_R) Y_R^T (Eq. updateC1), products into P (ldp = ldu).
  int c1_update(int64_t k, int q, int r0, int r1, double* P, int qs, cudaStream_t s) {
    if (!rq(k)) return 0;
    const int br = br_of(k), jr = jr_of(k);
    r1 = std::min<int>(r1, (int)std::min<int64_t>(w - br, m - k - br));
    if (r1 <= r0) return 0;
    double* C1 = R.A + (k + br + r0) + (k + w) * R.lda;
    int rc;
    if ((rc = R.prod_n(r1 - r0, br, jr, C1, R.lda, R.ws.Wv[q], R.ws.ldv, P, R.ws.ldu, qs, s))) return rc;
    return R.rank_k(r1 - r0, jr, br, P, R.ws.ldu, R.ws.Yv[q], R.ws.ldv, C1, R.lda, qs, s);
  }

  // Products of D for the two-sided update: Z_L = D^T W_L (ZT), X = D W_R + Y_L (Z_L^T W_R) (P).
  int d_products(int64_t k, int q, cudaStream_t s) {
    const int bl = bl_of(k), br = br_of(k), jl = jl_of(k), jr = jr_of(k);
    const bool l = lq(k), r = rq(k);
    if (jl < 1 || jr < 1 || !(l || r)) return 0;
    Ge2gbWs& ws = R.ws;
    const double* D = R.A + (k + w) + (k + w) * R.lda;
    int rc;
    if (l && (rc = R.prod_t(jr, bl, jl, D, R.lda, ws.Wu[q], ws.ldu, ws.ZT, ws.ldv, 0, s))) return rc;
    if (r) {
      if ((rc = R.prod_n(jl, br, jr, D, R.lda, ws.Wv[q], ws.ldv, ws.P, ws.ldu, 0, s))) return rc;
      if (l) {
        // S^T = W_R^T Z_L (br x bl), then X = Z_R + Y_L S
        if ((rc = R.prod_t(br, bl, jr, ws.Wv[q], ws.ldv, ws.ZT, ws.ldv, ws.MT, br, 0, s))) return rc;
        if ((rc = R.rank_k(jl, br, bl, ws.Yu[q], ws.ldu, ws.MT, br, ws.P, ws.ldu, 0, s))) return rc;
      }
    }
    return 0;
  }

  // D(r0:r1, c0:c1) += X Y_R^T + Y_L Z_L^T on those rows and columns (Eq. gebrd_2k).  With
  // the Ozaki precision one rank-(br + bl) update of [X | Y_L] and [Y_R | Z_L], balanced by a
  // power of two between the halves (X and Z_L carry the matrix's scale, |Y| <= 1).
  int d_rank(int64_t k, int q, int r0, int r1, int c0, int c1, int qs, cudaStream_t s, int max_ctas = 0) {
    const int bl = bl_of(k), br = br_of(k), jl = jl_of(k), jr = jr_of(k);
    const bool l = lq(k), r = rq(k);
    r1 = std::min(r1, jl);
    c1 = std::min(c1, jr);
    if (r1 <= r0 || c1 <= c0 || !(l || r)) return 0;
    Ge2gbWs& ws = R.ws;
    double* D = R.A + (k + w + r0) + (k + w + c0) * R.lda;
    const int M = r1 - r0, N = c1 - c0;
    if (R.o.precision == BANDRED_OZAKI && l && r) {
      using ozaki::Operand;
      prof::Scope sc(prof::kRank, s, 2.0 * M * N * (bl + br), 8.0 * (2.0 * M * N + (double)(M + N) * (bl + br)));
      Operand lo{ws.P + r0, ws.ldu, 0, br, ws.Yu[q] + r0, ws.ldu, 0, bl, M};
      Operand ro{ws.Yv[q] + c0, ws.ldv, 0, br, ws.ZT + c0, ws.ldv, 0, bl, N};
      int* sh = ws.sh + 0;
      // one balance per iteration serves every block of D (the exponents of the full X, Y_L)
      lo.sh = ro.sh = sh;
      lo.shsign = 1;
      ro.shsign = -1;
      const ozaki::Bufs rb = ozaki::carve(ws.ozr[qs], M, N, br + bl, 1);
      CK(ozaki::prepare(lo, ro, rb, s));
      CK(ozaki::rank_apply(M, N, br + bl, 1.0, D, R.lda, 0, N, 0, rb, R.status, R.o.limit_ns, s, max_ctas));
      return 0;
    }
    int rc;
    if (r && (rc = R.rank_k(M, N, br, ws.P + r0, ws.ldu, ws.Yv[q] + c0, ws.ldv, D, R.lda, qs, s, max_ctas))) return rc;
    if (l && (rc = R.rank_k(M, N, bl, ws.Yu[q] + r0, ws.ldu, ws.ZT + c0, ws.ldv, D, R.lda, qs, s, max_ctas)))
      return rc;
    return 0;
  }

  // The balance exponents of [X | Y_L] over all of D's rows (before any block of d_rank).
  int d_balance(int64_t k, int q, cudaStream_t s) {
    if (R.o.precision != BANDRED_OZAKI || !lq(k) || !rq(k) || jl_of(k) < 1 || jr_of(k) < 1) return 0;
    Ge2gbWs& ws = R.ws;
    const ozaki::Operand lo{ws.P, ws.ldu, 0, br_of(k), ws.Yu[q], ws.ldu, 0, bl_of(k), jl_of(k)};
    CK(ozaki::balance(lo, ws.sh, s));
    return 0;
  }
};

}  // namespace

// Auto (-1): V1 when 2b <= w; no look-ahead otherwise (at m = n = 8192, w = b = 64 the V2
// schedule measured 174 ms against 160 ms without: its two extra block updates of D cost
// more than the panels' overlap saves); 2 asks for V2 explicitly.
static int ge2bb_variant(const Options& o, int64_t w) {
  int la = o.lookahead;
  if (la < 0) la = (2 * o.b > w) ? 0 : 1;
  if (la == 0) return 0;
  if (la == 1 && 2 * o.b > w) la = 2;
  if (la == 2 && 2 * o.b <= w) la = 1;
  return la;
}

int ge2bb_run(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup, const Options& o,
              void* work, int* dev_status, cudaStream_t s) {
  Ge2bb G{};
  Ge2gb& R = G.R;
  R.m = m;
  R.n = n;
  R.w = w;
  R.A = A;
  R.lda = lda;
  R.tauq = tauq;
  R.taup = taup;
  R.o = o;
  R.sms = current_sms();
  R.ws = carve_ge2gb(work, std::max(m, n), std::max(m, n), w, o, R.sms, true);
  R.status = dev_status ? dev_status : R.ws.status;
  R.pmax = panel_max_ctas(R.sms, o);
  R.S = is_split(o) ? split::slices_of(o.precision) : 0;
  R.extra = 0;
  G.m = m;
  G.n = n;
  G.w = w;
  G.b = o.b;
  G.nlq = std::max<int64_t>(0, std::min(n, m - w));
  G.nrq = std::max<int64_t>(0, std::min(m, n - w));
  CK(cudaMemsetAsync(R.status, 0, sizeof(int), s));
  if (G.nlq > 0) CK(cudaMemsetAsync(tauq, 0, sizeof(double) * G.nlq, s));
  if (G.nrq > 0) CK(cudaMemsetAsync(taup, 0, sizeof(double) * G.nrq, s));
  const int b = o.b;
  const int64_t kend = std::max(G.nlq, G.nrq);
  const int la = o.lookahead == 0 ? 0 : ge2bb_variant(o, w);
  int rc;
  if (la == 0 || kend <= b) {
    for (int64_t k = 0; k < kend; k += b) {
      if ((rc = G.panels(k, 0, s))) return rc;
      if ((rc = G.b1_update(k, 0, 0, (int)w, R.ws.ZT, 0, s))) return rc;
      if ((rc = G.c1_update(k, 0, 0, (int)w, R.ws.P, 0, s))) return rc;
      if ((rc = G.d_products(k, 0, s))) return rc;
      if ((rc = G.d_balance(k, 0, s))) return rc;
      if ((rc = G.d_rank(k, 0, 0, (int)m, 0, (int)n, 0, s))) return rc;
    }
    return 0;
  }
  AuxStreams* ax = nullptr;
  if ((rc = aux_streams(&ax))) return rc;
  cudaStream_t sp = ax->panel;
  cudaEvent_t ev_fork = ax->ev[0], ev_panel = ax->ev[1];
  CK(cudaEventRecord(ev_fork, s));
  CK(cudaStreamWaitEvent(sp, ev_fork, 0));
  if ((rc = G.panels(0, 0, sp))) return rc;
  CK(cudaEventRecord(ev_panel, sp));
  int buf = 0;
  for (int64_t k = 0; k < kend; k += b, buf ^= 1) {
    const int64_t kn = k + b;
    const bool has_next = kn < kend;
    CK(cudaStreamWaitEvent(s, ev_panel, 0));  // the panels of iteration k are factored
    if (la == 1) {
      if (has_next) {
        CK(cudaEventRecord(ev_fork, s));  // iteration k - b's update is complete
        CK(cudaStreamWaitEvent(sp, ev_fork, 0));
        if ((rc = G.b1_update(k, buf, 0, b, R.ws.ZT2, 1, sp))) return rc;
        if ((rc = G.c1_update(k, buf, 0, b, R.ws.P2, 1, sp))) return rc;
        if ((rc = G.panels(kn, buf ^ 1, sp))) return rc;
        CK(cudaEventRecord(ev_panel, sp));
      }
      const int rest = has_next ? b : 0;
      if ((rc = G.b1_update(k, buf, rest, (int)w, R.ws.ZT, 0, s))) return rc;
      if ((rc = G.c1_update(k, buf, rest, (int)w, R.ws.P, 0, s))) return rc;
      if ((rc = G.d_products(k, buf, s))) return rc;
      if ((rc = G.d_balance(k, buf, s))) return rc;
      if ((rc = G.d_rank(k, buf, 0, (int)m, 0, (int)n, 0, s))) return rc;
      continue;
    }
    // V2
    if ((rc = G.b1_update(k, buf, 0, (int)w, R.ws.ZT2, 0, s))) return rc;
    if ((rc = G.c1_update(k, buf, 0, (int)w, R.ws.P2, 0, s))) return rc;
    if ((rc = G.d_products(k, buf, s))) return rc;
    if ((rc = G.d_balance(k, buf, s))) return rc;
    if (!has_next) {
      if ((rc = G.d_rank(k, buf, 0, (int)m, 0, (int)n, 0, s))) return rc;
      continue;
    }
    const int t = (int)(2 * b - w);
    // with the Ozaki precision the panel stream (its blocks of D, then the panels) holds P
    // SMs and D(t:, t:) the others, by the look-ahead model with the rank-(bl + br) update
    const int jn = std::max(G.jl_of(kn), G.jr_of(kn)), jd = std::max(G.jl_of(k), G.jr_of(k));
    const int P = o.precision == BANDRED_OZAKI && jn > 1
                      ? lookahead_panel_ctas(jn, b, jd, 2 * b, R.sms, o.panel_ctas, cluster_panels(o))
                      : 0;
    const int rest = P > 0 && P < R.sms ? R.sms - P : 0;
    CK(cudaEventRecord(ev_fork, s));
    CK(cudaStreamWaitEvent(sp, ev_fork, 0));
    if ((rc = G.d_rank(k, buf, 0, (int)m, 0, t, 1, sp, P))) return rc;  // D(:, 0:t)
    if ((rc = G.d_rank(k, buf, 0, t, t, (int)n, 1, sp, P))) return rc;  // D(0:t, t:)
    if ((rc = G.panels(kn, buf ^ 1, sp, P))) return rc;
    CK(cudaEventRecord(ev_panel, sp));
    if ((rc = G.d_rank(k, buf, t, (int)m, t, (int)n, 0, s, rest))) return rc;  // D(t:, t:)
  }
  CK(cudaEventRecord(ev_fork, sp));
  CK(cudaStreamWaitEvent(s, ev_fork, 0));
  return 0;
}

size_t ge2bb_workspace_bytes(int64_t m, int64_t n, int64_t w, const Options& o) {
  return carve_ge2gb(nullptr, std::max(m, n), std::max(m, n), w, o, current_sms(), true).bytes;
}

size_t ge2gb_workspace_bytes(int64_t m, int64_t n, int64_t w, const Options& o) {
  if (n > m) return align_up((size_t)m * n * sizeof(double)) + ge2gb_workspace_bytes(n, m, w, o);
  return carve_ge2gb(nullptr, m, n, w, o, current_sms()).bytes;
}

}  // namespace bandred
