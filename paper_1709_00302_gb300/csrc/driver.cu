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
#include "kernels.h"
#include "prof.h"

namespace bandred {

namespace {

constexpr size_t kAlign = 256;
constexpr int kMinPanelRows = 32;
constexpr int kMaxSplits = 128;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

thread_local char g_last_error[512] = "";

struct DeviceInfo {
  int sms = 0;
};

DeviceInfo& device_info(int dev) {
  static std::mutex mu;
  static DeviceInfo info[64];
  std::lock_guard<std::mutex> lock(mu);
  DeviceInfo& d = info[dev & 63];
  if (d.sms == 0) cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
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

int panel_max_ctas(int sms, const Options& o) {
  if (o.panel_ctas > 0) return std::min(o.panel_ctas, sms);
  return sms;
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
  o->b = d.b;
  o->lookahead = d.lookahead;
  o->precision = d.precision;
  o->slices = d.slices;
  o->panel_ctas = d.panel_ctas;
  o->limit_ns = (unsigned long long)(d.timeout_ms ? d.timeout_ms : 2000) * 1000000ull;
  o->debug = d.debug;
  return 0;
}

// Workspace of sy2sb (layout shared by sizing and carving).
struct Sy2sbWs {
  double *Y, *W, *X, *X2, *Z, *splitk, *part, *rowbuf, *part2;
  GridSync* gs;
  int* status;
  int64_t ld;
  size_t splitk_cap;
  size_t bytes;
};

static Sy2sbWs carve_sy2sb(void* work, int64_t n, int64_t w, const Options& o, int sms) {
  Carver c{static_cast<char*>(work)};
  Sy2sbWs ws{};
  const int64_t jmax = std::max<int64_t>(n - w, 1);
  const int64_t b = o.b;
  ws.ld = jmax;
  ws.Y = c.take<double>(jmax * b);
  ws.W = c.take<double>(jmax * b);
  ws.X = c.take<double>(jmax * b);
  ws.X2 = c.take<double>(b * b);
  ws.Z = c.take<double>(b * std::max<int64_t>(w, 1));
  ws.splitk_cap = (size_t)kMaxSplits * b * std::max<int64_t>(w, b);
  ws.splitk = c.take<double>(ws.splitk_cap);
  ws.part = c.take<double>(2 * (size_t)sms * (b + 1));
  ws.rowbuf = c.take<double>(2 * (size_t)b);
  ws.part2 = c.take<double>((size_t)sms);
  ws.gs = c.take<GridSync>(1);
  ws.status = c.take<int>(1);  // last piece: the short forms read it at bytes - 256
  ws.bytes = c.off;
  return ws;
}

struct Ge2gbWs {
  double *Yu, *Wu, *Yv, *Wv, *Z, *P, *splitk, *part, *rowbuf, *part2;
  GridSync* gs;
  int* status;
  int64_t ldu, ldv;
  size_t splitk_cap;
  size_t bytes;
};

static Ge2gbWs carve_ge2gb(void* work, int64_t m, int64_t n, const Options& o, int sms) {
  Carver c{static_cast<char*>(work)};
  Ge2gbWs ws{};
  const int64_t b = o.b;
  ws.ldu = std::max<int64_t>(m, 1);
  ws.ldv = std::max<int64_t>(n, 1);
  ws.Yu = c.take<double>(ws.ldu * b);
  ws.Wu = c.take<double>(ws.ldu * b);
  ws.Yv = c.take<double>(ws.ldv * b);
  ws.Wv = c.take<double>(ws.ldv * b);
  ws.Z = c.take<double>(b * ws.ldv);
  ws.P = c.take<double>(ws.ldu * b);
  ws.splitk_cap = (size_t)kMaxSplits * b * b * 4;
  ws.splitk = c.take<double>(ws.splitk_cap);
  ws.part = c.take<double>(2 * (size_t)sms * (b + 1));
  ws.rowbuf = c.take<double>(2 * (size_t)b);
  ws.part2 = c.take<double>((size_t)sms);
  ws.gs = c.take<GridSync>(1);
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
static int run_panel(double* A, int64_t rs, int64_t cs, int j, int bk, double* tau, double* Y, double* W,
                     int64_t ldy, double* part, double* rowbuf, double* part2, GridSync* gs, int* status,
                     const Options& o, int max_ctas, unsigned int extra, cudaStream_t s) {
  int G, R, Rp;
  bool w_smem = false;
  if (panel_geometry(j, bk, max_ctas, kMinPanelRows, &G, &R, &Rp, &w_smem) != 0) return BANDRED_ERR_UNSUPPORTED;
  PanelParams p{};
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
  p.part = part;
  p.rowbuf = rowbuf;
  p.part2 = part2;
  p.gs = gs;
  p.status = status;
  p.limit_ns = o.limit_ns;
  p.extra = extra;
  p.w_in_smem = w_smem;
  CK(launch_panel(p, G, s));
  return 0;
}

// ---------------------------------------------------------------------------------
// sy2sb: Section 2.1 loop.  Iteration k: panel A0 = A(k+w:n, k:k+bk) (Eq. updateA0),
// A1 = A(k+w:n, k+bk:k+w) := A1 + Y (W^T A1) (Eq. updateA1), and the two-sided update of
// A2 = A(k+w:n, k+w:n) through X1 = A2 W, X2 = X1^T W / 2, X3 = X1 + Y X2,
// A2 += X3 Y^T + Y X3^T (Eqs. updateA2symm .. updateA2syr2k).
int sy2sb_run(int64_t n, int64_t w, double* A, int64_t lda, double* tau, const Options& o, void* work,
              int* dev_status, cudaStream_t s) {
  const int sms = current_sms();
  Sy2sbWs ws = carve_sy2sb(work, n, w, o, sms);
  int* status = dev_status ? dev_status : ws.status;
  CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  const int64_t nref = n - w;
  if (nref <= 0) return 0;
  CK(cudaMemsetAsync(tau, 0, sizeof(double) * nref, s));
  const int b = o.b;
  const int64_t ld = ws.ld;
  const int pmax = panel_max_ctas(sms, o);
  unsigned int extra = o.debug ? 1u : 0u;
  for (int64_t k = 0; k <= n - w - 2; k += b) {
    const int bk = (int)std::min<int64_t>(b, n - w - 1 - k);
    const int64_t r0 = k + w;
    const int j = (int)(n - r0);
    int rc;
    {
      prof::Scope sc(prof::kPanel, s, panel_flops(j, bk), panel_bytes(j, bk));
      rc = run_panel(A + r0 + k * lda, 1, lda, j, bk, tau + k, ws.Y, ws.W, ld, ws.part, ws.rowbuf, ws.part2, ws.gs,
                     status, o, pmax, extra, s);
    }
    if (rc) return rc;
    extra = 0;
    const int na1 = (int)(w - bk);
    if (na1 > 0) {
      double* A1 = A + r0 + (k + bk) * lda;
      const int sp = choose_splits(bk, na1, j, ws.splitk_cap, sms);
      prof::Scope sc(prof::kGemm, s, 4.0 * j * na1 * bk, 8.0 * (2.0 * j * na1 + 2.0 * j * bk));
      CK(gemm_f64(bk, na1, j, 1.0, MatView{ws.W, ld, 1}, MatView{A1, 1, lda}, 0.0, ws.Z, bk, sp, ws.splitk, s));
      CK(gemm_f64(j, na1, bk, 1.0, MatView{ws.Y, 1, ld}, MatView{ws.Z, 1, bk}, 1.0, A1, lda, 1, nullptr, s));
    }
    double* A2 = A + r0 + r0 * lda;
    {
      prof::Scope sc(prof::kSymm, s, symm_flops(j, bk), symm_bytes(j, bk));
      CK(symm_lower_f64(j, bk, A2, lda, ws.W, ld, ws.X, ld, s));
    }
    {
      prof::Scope sc(prof::kGemm, s, 4.0 * j * bk * bk, 8.0 * 4.0 * j * bk);
      const int sp = choose_splits(bk, bk, j, ws.splitk_cap, sms);
      CK(gemm_f64(bk, bk, j, 0.5, MatView{ws.X, ld, 1}, MatView{ws.W, 1, ld}, 0.0, ws.X2, bk, sp, ws.splitk, s));
      CK(gemm_f64(j, bk, bk, 1.0, MatView{ws.Y, 1, ld}, MatView{ws.X2, 1, bk}, 1.0, ws.X, ld, 1, nullptr, s));
    }
    {
      prof::Scope sc(prof::kSyr2k, s, syr2k_flops(j, 0, j, bk), syr2k_bytes(j, 0, j, bk));
      CK(syr2k_lower_f64(j, bk, A2, lda, ws.X, ld, ws.Y, ld, 0, j, s));
    }
  }
  return 0;
}

size_t sy2sb_workspace_bytes(int64_t n, int64_t w, const Options& o) {
  return carve_sy2sb(nullptr, n, w, o, current_sms()).bytes;
}

// ---------------------------------------------------------------------------------
// ge2gb: Section 3.1 loop.  Iteration k: QR of B = A(k:m, k:k+bk) (Eq. updateB),
// E = A(k:m, k+bk:n) += Y_U (W_U^T E) (Eq. updateCD), LQ of C = A(k:k+bkr, k+w:n)
// (Eq. updateC), D = A(k+bkr:m, k+w:n) += (D W_V) Y_V^T (Eq. updateD).
int ge2gb_run(int64_t m, int64_t n, int64_t w, double* A, int64_t lda, double* tauq, double* taup,
              const Options& o, void* work, int* dev_status, cudaStream_t s) {
  const int sms = current_sms();
  Ge2gbWs ws = carve_ge2gb(work, m, n, o, sms);
  int* status = dev_status ? dev_status : ws.status;
  CK(cudaMemsetAsync(status, 0, sizeof(int), s));
  if (n <= 0) return 0;
  CK(cudaMemsetAsync(tauq, 0, sizeof(double) * n, s));
  if (n - w > 0) CK(cudaMemsetAsync(taup, 0, sizeof(double) * (n - w), s));
  const int b = o.b;
  const int pmax = panel_max_ctas(sms, o);
  unsigned int extra = o.debug ? 1u : 0u;
  for (int64_t k = 0; k < n; k += b) {
    const int bk = (int)std::min<int64_t>(b, n - k);
    const int j = (int)(m - k);
    int rc;
    {
      prof::Scope sc(prof::kPanel, s, panel_flops(j, bk), panel_bytes(j, bk));
      rc = run_panel(A + k + k * lda, 1, lda, j, bk, tauq + k, ws.Yu, ws.Wu, ws.ldu, ws.part, ws.rowbuf, ws.part2,
                     ws.gs, status, o, pmax, extra, s);
    }
    if (rc) return rc;
    extra = 0;
    const int ncol = (int)(n - k - bk);
    if (ncol > 0) {
      double* E = A + k + (k + bk) * lda;
      const int sp = choose_splits(bk, ncol, j, ws.splitk_cap, sms);
      prof::Scope sc(prof::kGemm, s, 4.0 * j * ncol * bk, 8.0 * (2.0 * j * ncol + 2.0 * j * bk));
      CK(gemm_f64(bk, ncol, j, 1.0, MatView{ws.Wu, ws.ldu, 1}, MatView{E, 1, lda}, 0.0, ws.Z, bk, sp, ws.splitk,
                  s));
      CK(gemm_f64(j, ncol, bk, 1.0, MatView{ws.Yu, 1, ws.ldu}, MatView{ws.Z, 1, bk}, 1.0, E, lda, 1, nullptr, s));
    }
    const int64_t bkr = std::min<int64_t>(bk, n - w - 1 - k);
    if (bkr > 0) {
      const int jr = (int)(n - k - w);
      {
        prof::Scope sc(prof::kPanel, s, panel_flops(jr, (int)bkr), panel_bytes(jr, (int)bkr));
        rc = run_panel(A + k + (k + w) * lda, lda, 1, jr, (int)bkr, taup + k, ws.Yv, ws.Wv, ws.ldv, ws.part,
                       ws.rowbuf, ws.part2, ws.gs, status, o, pmax, 0u, s);
      }
      if (rc) return rc;
      const int nrow = (int)(m - k - bkr);
      if (nrow > 0) {
        double* D = A + (k + bkr) + (k + w) * lda;
        const int sp = choose_splits(nrow, (int)bkr, jr, ws.splitk_cap, sms);
        prof::Scope sc(prof::kGemm, s, 4.0 * nrow * jr * bkr, 8.0 * (2.0 * nrow * jr + 2.0 * nrow * bkr));
        CK(gemm_f64(nrow, (int)bkr, jr, 1.0, MatView{D, 1, lda}, MatView{ws.Wv, 1, ws.ldv}, 0.0, ws.P, ws.ldu, sp,
                    ws.splitk, s));
        CK(gemm_f64(nrow, jr, (int)bkr, 1.0, MatView{ws.P, 1, ws.ldu}, MatView{ws.Yv, ws.ldv, 1}, 1.0, D, lda, 1,
                    nullptr, s));
      }
    }
  }
  return 0;
}

size_t ge2gb_workspace_bytes(int64_t m, int64_t n, int64_t w, const Options& o) {
  return carve_ge2gb(nullptr, m, n, o, current_sms()).bytes;
}

}  // namespace bandred
