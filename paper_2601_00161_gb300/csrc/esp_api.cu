// C ABI of the ESP long-range step (declared in include/esp.h): plan construction on
// the host in FP64 and the per-step launch sequence
//   bin -> scan -> scatter -> spread -> cuFFT R2C -> scale+reduce [-> cuFFT C2R -> gather]
// on the plan's stream.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "esp.h"
#include "esp_kernels.cuh"
#include "esp_pswf.h"

namespace {

thread_local std::string g_plan_error;

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct esp_plan_s {
  // configuration
  bool fp64 = true;
  bool io_double = true;
  bool bf16 = false;  // the potential grid is stored in BF16 (ESP_BF16_GRID)
  int64_t n = 0;
  int M[3] = {0, 0, 0};
  int H2 = 0;
  int P = 0;
  double c = 0.0, rc = 0.0;
  int device = 0;
  cudaStream_t stream = nullptr;
  // cell
  double h[9] = {0};     // row-major h[r][c]
  double hinv[9] = {0};  // row-major
  double V = 0.0;
  // PSWF constants
  esp::Prolate pswf;
  double A = 0.0;       // 4 pi / psi_0(0)
  double selfc = 0.0;   // psi_0(0) / (2 C_0 r_c)
  double Xbg = 0.0;     // r_c^2/2 - int_0^{r_c} r phi_0(r) dr
  int deg = 0, rdeg = 0;
  double fit_err = 0.0, rfit_err = 0.0;
  // geometry
  esp::TileGeom tg{};
  esp::ScaleGeom sg{};
  esp::GatherGeom gg{};
  int ntiles = 0;
  esp::XGeom xg{};       // the transform along axis 0 fused with the scaling
  int xblocks = 0;       // its CTAs: column groups
  // plane transforms over (i1, i2): the library's pruned kernels into the box of the
  // sphere (box_mode), else cuFFT into the full half spectrum
  esp::PlaneGeom pg{};
  bool box_mode = false;
  void* d_pbox = nullptr;  // planes transformed, the input of k_xfft (kept for forces)
  void* d_ptw = nullptr;   // M1 then M2 roots (compute type)
  void* d_phi16 = nullptr; // the potential grid in BF16 (ESP_BF16_GRID)
  int xactive = 0;       // groups whose lines may meet the sphere (ordered first)
  int* d_xorder = nullptr;           // group order, active first
  unsigned char* d_xcol = nullptr;   // per column: line may meet the sphere
  int* h_xorder = nullptr;           // pinned staging of the two
  unsigned char* h_xcol = nullptr;
  // the final sum of the transform's per-CTA partials runs on a branch of its own
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_start = nullptr, ev_zero = nullptr;
  int bin_blocks = 0;
  int spread_blocks = 0, gather_blocks = 0;
  int sms = 152;  // SMs of the plan's device
  // device buffers
  void* d_wtab = nullptr;
  void* d_radtab = nullptr;
  void* d_invw2 = nullptr;
  void* d_grid = nullptr;
  void* d_spec = nullptr;
  void* d_spec2 = nullptr;  // scaled half spectrum, input of the plane C2R (cleared per step)
  void* d_xtw = nullptr;  // M0 roots e^{-2 pi i m / M0} (compute type)
  // atoms binned by tile (esp::Bins): slot arrays, counters, overflow list, control words
  esp::Bins bins{};
  double* d_binpart = nullptr;  // per binning block: sum q, sum q^2, skipped atoms
  double* d_accum = nullptr;
  double* d_partials = nullptr;
  void* d_io_pos = nullptr;
  void* d_io_q = nullptr;
  void* d_io_f = nullptr;
  double* h_accum = nullptr;  // pinned
  // plane transforms over (i1, i2) for every i0 (R2C / C2R, batched) of the force step,
  // whose transform along i0 is k_xfft; fwd3: the full 3D R2C of the energy and pressure
  // step (the spectrum is kept); inv3: the full 3D C2R of one field (on first use)
  cufftHandle fwd = 0, inv = 0, fwd3 = 0, inv3 = 0;
  bool have_fwd = false, have_inv = false, have_fwd3 = false, have_inv3 = false;
  bool spectrum_kept = false;
  // CUDA graph of the last esp_step (re-captured when its arguments or the cell change)
  bool use_graph = true;
  cudaGraphExec_t graph_exec = nullptr;
  const void* g_pos = nullptr;
  const void* g_q = nullptr;
  void* g_f = nullptr;
  double* g_acc = nullptr;
  bool g_prof = false;
  // near part (allocated by the first esp_near call; the cell list follows the cell)
  esp::NearGeom ng{};
  int near_cells_alloc = 0;
  int near_ndeg = 0;
  void* d_neartab = nullptr;
  int* d_ncount = nullptr;  // atoms per cell (zero between calls)
  int* d_ncoff = nullptr;   // exclusive offsets (cells + 1)
  int* d_ncell = nullptr;
  int* d_nrank = nullptr;
  void* d_nxq_tmp = nullptr;
  void* d_nxq = nullptr;
  int* d_nidx = nullptr;
  void* d_noff = nullptr;  // displacements of a block's neighbourhood cells
  // field variants (allocated on first use): up to 6 half spectra and 6 real grids, batched
  // inverse transforms for 3 and 6 fields
  void* d_fspec = nullptr;
  void* d_fgrid = nullptr;
  cufftHandle finv3 = 0, finv6 = 0;
  bool have_finv3 = false, have_finv6 = false;
  // per-stage CUDA events (esp_profile)
  bool profiling = false;
  cudaEvent_t ev[16] = {};
  bool ev_used[16] = {};
  std::string err;
};

namespace {

int fail(esp_plan_t p, int code, const std::string& msg) {
  if (p)
    p->err = msg;
  else
    g_plan_error = msg;
  return code;
}

int cuda_fail(esp_plan_t p, cudaError_t e, const char* what) {
  return fail(p, ESP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define ESP_CUDA(p, call)                                          \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail((p), e_, #call);       \
  } while (0)

#define ESP_CUFFT(p, call)                                                          \
  do {                                                                              \
    cufftResult r_ = (call);                                                        \
    if (r_ != CUFFT_SUCCESS)                                                        \
      return fail((p), ESP_ERR_CUFFT, std::string(#call) + " failed, cufftResult " + \
                                           std::to_string((int)r_));                \
  } while (0)

// h from the column-major cell[9] (columns are the cell vectors); checks det h > 0.
int set_cell_matrix(esp_plan_t p, const double cell[9], double h[9], double hinv[9],
                    double* V) {
  if (!cell) return fail(p, ESP_ERR_ARG, "cell is NULL");
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(cell[i])) return fail(p, ESP_ERR_CELL, "non-finite cell entry");
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) h[3 * r + c] = cell[3 * c + r];
  const double c00 = h[4] * h[8] - h[5] * h[7];
  const double c01 = h[5] * h[6] - h[3] * h[8];
  const double c02 = h[3] * h[7] - h[4] * h[6];
  const double det = h[0] * c00 + h[1] * c01 + h[2] * c02;
  if (!(det > 0.0) || !std::isfinite(det)) return fail(p, ESP_ERR_CELL, "det h must be positive");
  const double id = 1.0 / det;
  hinv[0] = c00 * id;
  hinv[1] = (h[2] * h[7] - h[1] * h[8]) * id;
  hinv[2] = (h[1] * h[5] - h[2] * h[4]) * id;
  hinv[3] = c01 * id;
  hinv[4] = (h[0] * h[8] - h[2] * h[6]) * id;
  hinv[5] = (h[2] * h[3] - h[0] * h[5]) * id;
  hinv[6] = c02 * id;
  hinv[7] = (h[1] * h[6] - h[0] * h[7]) * id;
  hinv[8] = (h[0] * h[4] - h[1] * h[3]) * id;
  *V = det;
  return ESP_OK;
}

// Every mode with |k| <= K = c/r_c has |m_d| = |h_d . k| / 2pi <= |h_d| K / 2pi; require
// that bound below M_d/2 so no such mode reaches the Nyquist index.
int check_grid(esp_plan_t p, const double h[9], const int M[3], double c, double rc,
               int mmax[3]) {
  const double K = c / rc;
  for (int d = 0; d < 3; ++d) {
    const double len = std::sqrt(h[d] * h[d] + h[3 + d] * h[3 + d] + h[6 + d] * h[6 + d]);
    const double bound = len * K / (2.0 * M_PI);
    if (!(bound < 0.5 * M[d])) {
      char buf[200];
      std::snprintf(buf, sizeof buf,
                    "grid too coarse in dimension %d: need M > |h_d| c / (pi r_c) = %.3f", d,
                    2.0 * bound);
      return fail(p, ESP_ERR_GRID, buf);
    }
    mmax[d] = std::min((int)std::floor(bound), (M[d] - 1) / 2);
  }
  return ESP_OK;
}

void update_cell_constants(esp_plan_t p) {
  std::memcpy(p->tg.hinv, p->hinv, sizeof p->hinv);
  for (int i = 0; i < 9; ++i) p->tg.hinvf[i] = (float)p->hinv[i];
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) {
      const double A = (double)p->M[d] * p->hinv[3 * d + e];
      p->tg.Ahi[3 * d + e] = (float)A;
      p->tg.Alo[3 * d + e] = (float)(A - (double)(float)A);
    }
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 3; ++a) {
      p->sg.b[3 * d + a] = 2.0 * M_PI * p->hinv[3 * d + a];
      p->sg.bf[3 * d + a] = (float)p->sg.b[3 * d + a];
    }
  const double Mtot = (double)p->M[0] * p->M[1] * p->M[2];
  p->sg.scale = 1.0 / (2.0 * p->V * Mtot * Mtot);
  p->sg.scalef = (float)p->sg.scale;
  p->gg.g = p->tg;
  p->gg.fscale = 1.0 / (p->V * Mtot * Mtot);
  p->gg.fscalef = (float)p->gg.fscale;
}

// Column groups of the transform along axis 0 for the current cell: a column (m1, m2) is
// active when its line k = m0 b_0 + v (v = m1 b_1 + m2 b_2) may enter the sphere |k| <= K:
// |m1| <= mmax1, m2 <= mmax2 and the squared distance |v|^2 - (v.b_0)^2 / |b_0|^2 of the
// line from the origin at most K^2 (1 + 1e-6).  Groups with an active column come first.
// The staging copy waits for the stream, so a step still reading the old order is done.
int update_xfft_tasks(esp_plan_t p) {
  const esp::ScaleGeom& s = p->sg;
  const esp::XGeom& x = p->xg;
  const double* b = s.b;
  const double bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  ESP_CUDA(p, cudaStreamSynchronize(p->stream));
  const int NC = 1 << x.lognc;
  int na = 0, ni = p->xblocks - 1;
  for (int gi = 0; gi < p->xblocks; ++gi) {
    bool any = false;
    for (int c = 0; c < NC; ++c) {
      const int f = gi * NC + c;
      if (f >= x.ncol) break;
      const int b1 = f / x.nb2, m2 = f % x.nb2;
      const int m1 = (2 * b1 <= x.nb1) ? b1 : b1 - x.nb1;
      bool act = false;
      if (std::abs(m1) <= s.mmax[1] && m2 <= s.mmax[2]) {
        const double vx = m1 * b[3] + m2 * b[6], vy = m1 * b[4] + m2 * b[7], vz = m1 * b[5] + m2 * b[8];
        const double vb = vx * b[0] + vy * b[1] + vz * b[2];
        act = vx * vx + vy * vy + vz * vz - vb * vb / bb <= s.K2 * (1.0 + 1e-6) + 1e-300;
      }
      p->h_xcol[f] = act ? 1 : 0;
      any = any || act;
    }
    // active groups from the front, the others from the back
    if (any)
      p->h_xorder[na++] = gi;
    else
      p->h_xorder[ni--] = gi;
  }
  // no active group (no mode inside the sphere): one group still writes the zero sums
  p->xactive = std::max(na, 1);
  if (na == 0) std::reverse(p->h_xorder, p->h_xorder + p->xblocks);
  ESP_CUDA(p, cudaMemcpyAsync(p->d_xorder, p->h_xorder, sizeof(int) * p->xblocks,
                              cudaMemcpyHostToDevice, p->stream));
  ESP_CUDA(p, cudaMemcpyAsync(p->d_xcol, p->h_xcol, (size_t)x.ncol, cudaMemcpyHostToDevice,
                              p->stream));
  return ESP_OK;
}

template <typename R>
std::vector<R> to_type(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

int upload(esp_plan_t p, void** dst, const std::vector<double>& src) {
  const size_t es = p->fp64 ? 8 : 4;
  ESP_CUDA(p, cudaMalloc(dst, std::max<size_t>(src.size(), 1) * es));
  if (p->fp64) {
    ESP_CUDA(p, cudaMemcpy(*dst, src.data(), src.size() * es, cudaMemcpyHostToDevice));
  } else {
    std::vector<float> f = to_type<float>(src);
    ESP_CUDA(p, cudaMemcpy(*dst, f.data(), f.size() * es, cudaMemcpyHostToDevice));
  }
  return ESP_OK;
}

// Window polynomials (Sec. 4.3): for stencil point p and t in [0,1) the window value is
// psi_0(u) with u = 2 (p + 1 - P/2 - t) / P; coefficients of (t - 1/2)^k, laid out
// [w: k * P + p][dw: (deg+1) * P + k * P + p].  The degree is fixed per compute type
// (kDegF32 / kDegF64, so that the kernels keep a lane's coefficients in registers); the
// plan fails if that degree does not reach the precision's tolerance, which happens only
// for a stencil far too narrow for c.
int build_window_tables(esp_plan_t p, std::vector<double>& tab) {
  const esp::Prolate& pr = p->pswf;
  const int P = p->P;
  const double tol = p->fp64 ? 1e-14 : 5e-8;
  const int deg = p->fp64 ? esp::kDegF64 : esp::kDegF32;
  double dmax = 0.0;
  for (int i = 0; i <= 200; ++i) dmax = std::max(dmax, std::fabs(pr.deriv(-1.0 + i / 100.0)));
  tab.assign(2 * (deg + 1) * P, 0.0);
  double err = 0.0;
  std::vector<double> coef(deg + 1);
  for (int pp = 0; pp < P; ++pp) {
    auto u_of = [P, pp](double t) { return 2.0 * (pp + 1.0 - 0.5 * P - t) / P; };
    double e1 = esp::fit_piece([&](double t) { return pr.eval(u_of(t)); }, 0.0, 1.0, deg,
                               coef.data());
    for (int k = 0; k <= deg; ++k) tab[k * P + pp] = coef[k];
    double e2 = esp::fit_piece([&](double t) { return pr.deriv(u_of(t)); }, 0.0, 1.0, deg,
                               coef.data());
    for (int k = 0; k <= deg; ++k) tab[(deg + 1) * P + k * P + pp] = coef[k];
    err = std::max(err, std::max(e1 / pr.psi_at_0, e2 / dmax));
  }
  p->deg = deg;
  p->fit_err = err;
  if (err > tol) {
    char buf[200];
    std::snprintf(buf, sizeof buf,
                  "window polynomial fit error %.2e exceeds %.0e: stencil P = %d too narrow "
                  "for c = %.3f",
                  err, tol, P, p->c);
    return fail(p, ESP_ERR_ARG, buf);
  }
  return ESP_OK;
}

// Near kernel on u = r / r_c in [0, 1], kRadialPieces pieces in (u - centre): 1 - phi_0(u)
// and F_N(u) = 1 - phi_0(u) + u psi_0(u) / C_0, phi_0(u) = (1 / C_0) int_0^u psi_0 from the
// Legendre series term by term (Sec. 3.1, eqs. (decomposition), (mathFN)).
int build_near_tables(esp_plan_t p, std::vector<double>& tab) {
  const esp::Prolate& pr = p->pswf;
  const double tol = p->fp64 ? 3e-15 : 2e-8;
  const int NR = esp::kRadialPieces;
  auto phi0 = [&](double u) { return pr.integral(u) / pr.C0; };
  auto g1 = [&](double u) { return 1.0 - phi0(u); };
  auto g2 = [&](double u) { return 1.0 - phi0(u) + u * pr.eval(u) / pr.C0; };
  for (int deg = 6; deg <= esp::kMaxDeg; ++deg) {
    tab.assign(2 * NR * (deg + 1), 0.0);
    std::vector<double> coef(deg + 1);
    double err = 0.0;
    for (int j = 0; j < NR; ++j) {
      const double lo = (double)j / NR, hi = (double)(j + 1) / NR;
      double e1 = esp::fit_piece(g1, lo, hi, deg, coef.data());
      for (int k = 0; k <= deg; ++k) tab[j * (deg + 1) + k] = coef[k];
      double e2 = esp::fit_piece(g2, lo, hi, deg, coef.data());
      for (int k = 0; k <= deg; ++k) tab[(NR + j) * (deg + 1) + k] = coef[k];
      err = std::max(err, std::max(e1, e2));  // both functions are 1 at u = 0
    }
    if (err <= tol || deg == esp::kMaxDeg) {
      if (err > (p->fp64 ? 1e-14 : 5e-8))
        return fail(p, ESP_ERR_ARG, "near-kernel polynomial fit did not converge");
      p->near_ndeg = deg;
      return ESP_OK;
    }
  }
  return ESP_OK;
}

// Radial psi_0 and psi_0' on x in [0, 1] (the Fourier kernel of eq. (UF) and its
// derivative in eq. (Far)), kRadialPieces pieces, coefficients of (x - centre)^k.
int build_radial_tables(esp_plan_t p, std::vector<double>& tab) {
  const esp::Prolate& pr = p->pswf;
  const double tol = p->fp64 ? 3e-15 : 2e-8;  // converged fits stop early
  const int NR = esp::kRadialPieces;
  double dmax = 0.0;
  for (int i = 0; i <= 100; ++i) dmax = std::max(dmax, std::fabs(pr.deriv(i / 100.0)));
  for (int deg = 6; deg <= esp::kMaxDeg; ++deg) {
    tab.assign(2 * NR * (deg + 1), 0.0);
    std::vector<double> coef(deg + 1);
    double err = 0.0;
    for (int j = 0; j < NR; ++j) {
      const double lo = (double)j / NR, hi = (double)(j + 1) / NR;
      double e1 = esp::fit_piece([&](double x) { return pr.eval(x); }, lo, hi, deg, coef.data());
      for (int k = 0; k <= deg; ++k) tab[j * (deg + 1) + k] = coef[k];
      double e2 = esp::fit_piece([&](double x) { return pr.deriv(x); }, lo, hi, deg, coef.data());
      for (int k = 0; k <= deg; ++k) tab[(NR + j) * (deg + 1) + k] = coef[k];
      err = std::max(err, std::max(e1 / pr.psi_at_0, e2 / std::max(dmax, 1e-300)));
    }
    if (err <= tol || deg == esp::kMaxDeg) {
      p->rdeg = deg;
      p->rfit_err = err;
      if (err > (p->fp64 ? 1e-14 : 5e-8))
        return fail(p, ESP_ERR_ARG, "radial polynomial fit did not converge");
      return ESP_OK;
    }
  }
  return ESP_OK;
}

// 1 / what_d(m)^2 with what_d(m) = int w_d(u) e^{-2 pi i m u} du
//                                = omega_d int_{-1}^{1} psi_0(t) cos(2 pi m omega_d t) dt
// (Sec. 4.2), evaluated here by Gauss-Legendre quadrature of the integral itself.
void build_invw2(esp_plan_t p, std::vector<double>& out) {
  const esp::Prolate& pr = p->pswf;
  std::vector<double> x, w;
  esp::gauss_legendre(160 + (int)std::ceil(2.0 * p->c), x, w);
  std::vector<double> fx(x.size());
  for (size_t i = 0; i < x.size(); ++i) fx[i] = pr.eval(x[i]) * w[i];
  out.clear();
  const int len[3] = {p->M[0], p->M[1], p->H2};
  for (int d = 0; d < 3; ++d) {
    const double om = p->P / (2.0 * p->M[d]);
    for (int i = 0; i < len[d]; ++i) {
      const int m = (d < 2 && 2 * i > p->M[d]) ? i - p->M[d] : i;
      double s = 0.0;
      for (size_t k = 0; k < x.size(); ++k) s += fx[k] * std::cos(2.0 * M_PI * m * om * x[k]);
      const double wh = om * s;
      out.push_back(wh != 0.0 ? 1.0 / (wh * wh) : 0.0);
    }
  }
}

void release(esp_plan_t p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  void* bufs[] = {p->d_wtab,      p->d_radtab,    p->d_invw2,    p->d_grid,      p->d_spec,  p->d_spec2, p->d_xtw, p->d_xorder, p->d_xcol,
                  p->d_pbox,      p->d_ptw,       p->d_phi16,
                  p->bins.count,  p->bins.tcount, p->bins.tq,    p->bins.lb,     p->bins.idx, p->bins.otq, p->bins.ob, p->bins.oidx,
                  p->bins.ctrl,   p->bins.hq,     p->d_binpart,   p->d_accum,   p->d_partials,
                  p->d_io_pos,    p->d_io_q,     p->d_io_f,
                  p->d_neartab,   p->d_ncount,    p->d_ncoff,    p->d_ncell,     p->d_nrank,
                  p->d_nxq_tmp,   p->d_nxq,       p->d_nidx,     p->d_noff,      p->d_fspec,     p->d_fgrid};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (p->h_accum) cudaFreeHost(p->h_accum);
  if (p->h_xorder) cudaFreeHost(p->h_xorder);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_zero) cudaEventDestroy(p->ev_zero);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->h_xcol) cudaFreeHost(p->h_xcol);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  for (cudaEvent_t e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->have_fwd) cufftDestroy(p->fwd);
  if (p->have_inv) cufftDestroy(p->inv);
  if (p->have_inv3) cufftDestroy(p->inv3);
  if (p->have_fwd3) cufftDestroy(p->fwd3);
  if (p->have_finv3) cufftDestroy(p->finv3);
  if (p->have_finv6) cufftDestroy(p->finv6);
  delete p;
}

unsigned int magic_of(unsigned int d) {
  return (unsigned int)((((unsigned long long)1 << 32) + d - 1) / d);
}

// Passes of a mixed-radix transform of length n: radices 8, 4, 2, 3, 5, 7, then the other
// prime factors; ns_magic[k] = ceil(2^32 / Ns), Ns the product of the radices before pass k.
bool radix_plan(int n, int* radix, unsigned int* ns_magic, int* npass) {
  int np = 0;
  auto push = [&](int r) {
    if (np < esp::kMaxPass) radix[np] = r;
    ++np;
    n /= r;
  };
  while (n % 8 == 0) push(8);
  if (n % 4 == 0) push(4);
  if (n % 2 == 0) push(2);
  for (int r : {3, 5, 7})
    while (n % r == 0) push(r);
  for (int r = 11; (int64_t)r * r <= n; r += 2)
    while (n % r == 0) push(r);
  if (n > 1) push(n);
  if (np > esp::kMaxPass) return false;
  *npass = np;
  for (int k = 0, ns = 1; k < np; ns *= radix[k], ++k) ns_magic[k] = magic_of((unsigned)ns);
  return true;
}

// Layout of the transform along the first axis and the plane transforms for the current
// cell.  The plane kernels keep only the box of the sphere (|m1| <= mmax1, m2 <= mmax2);
// when their shared memory would exceed the budget, cuFFT transforms the planes into the
// full half spectrum instead.  Either way the sizes stay within the buffers allocated
// for the full layout.
int setup_planes(esp_plan_t p) {
  esp::PlaneGeom& pg = p->pg;
  const int M1 = p->M[1], M2 = p->M[2];
  pg.M0 = p->M[0];
  pg.M1 = M1;
  pg.M2 = M2;
  pg.mmax1 = p->sg.mmax[1];
  pg.nb1 = 2 * p->sg.mmax[1] + 1;
  pg.nb2 = p->sg.mmax[2] + 1;
  pg.npairs = (M1 + 1) / 2;
  pg.m2_magic = magic_of((unsigned)M2);
  pg.nb2_magic = magic_of((unsigned)pg.nb2);
  bool ok = radix_plan(M2, pg.a.radix, pg.a.ns_magic, &pg.a.npass) &&
            radix_plan(M1, pg.b.radix, pg.b.ns_magic, &pg.b.npass);
  pg.a.n = M2;
  pg.b.n = M1;
  pg.b.nc = pg.nb2 | 1;
  pg.b.nc_magic = magic_of((unsigned)pg.b.nc);
  const size_t ce = p->fp64 ? 16 : 8;
  const size_t budget = 200 * 1024;
  int pb = std::min(32, pg.npairs + (pg.npairs & 1));
  pb += pb & 1;
  for (; pb >= 2; pb -= 2) {
    pg.pairs_b = pb;
    pg.a.nc = pb | 1;
    if (esp::plane_smem_bytes(p->fp64, pg) <= budget) break;
  }
  ok = ok && pb >= 2;
  if (ok) {
    pg.a.nc_magic = magic_of((unsigned)pg.a.nc);
    // every magic division stays exact: x d < 2^32 for the largest dividend x
    const uint64_t lim = (uint64_t)1 << 32;
    ok = (uint64_t)M2 * pg.a.nc * pg.a.nc < lim && (uint64_t)M1 * pg.b.nc * pg.b.nc < lim &&
         (uint64_t)M2 * pg.a.nc * M2 < lim && (uint64_t)pg.nb2 * pg.a.nc * pg.nb2 < lim &&
         (uint64_t)pg.nb1 * pg.nb2 * pg.nb2 < lim;
  }
  (void)ce;
  esp::XGeom& x = p->xg;
  if (!ok && p->bf16)
    return fail(p, ESP_ERR_ARG, "ESP_BF16_GRID needs the library's plane transforms, which "
                                "do not fit this grid");
  p->box_mode = ok;
  if (ok) {
    x.nb1 = pg.nb1;
    x.nb2 = pg.nb2;
    const cudaError_t e = esp::configure_planes(p->fp64, esp::plane_smem_bytes(p->fp64, pg));
    if (e != cudaSuccess) return cuda_fail(p, e, "cudaFuncSetAttribute (plane transforms)");
  } else {
    x.nb1 = M1;
    x.nb2 = p->H2;
  }
  x.ncol = x.nb1 * x.nb2;
  p->xblocks = esp::xfft_blocks(x);
  return ESP_OK;
}

// Tile geometry of spread and gather (p->M, p->P, p->fp64, p->deg and p->pswf set).  A
// tile holds T0 x T1 x T2 stencil bases; the CTA working on it owns the padded block
// (T + P - 1)^3.  T2 is a multiple of 4 so padded rows move as aligned float4 when M2 is
// too.  Many small tiles keep the persistent CTAs of spread and gather busy to the end.
int setup_tile_geom(esp_plan_t p) {
  esp::TileGeom& g = p->tg;
  const int w = p->P;
  for (int d = 0; d < 3; ++d) g.M[d] = p->M[d];
  g.P = w;
  {
    int Tc[3], E3p, vol;
    esp::tile_shape(w, Tc, &E3p, &vol);
    for (int d = 0; d < 3; ++d) g.T[d] = std::min(Tc[d], p->M[d]);
    g.E3p = E3p;
  }
  p->ntiles = 1;
  for (int d = 0; d < 3; ++d) {
    g.nt[d] = (p->M[d] + g.T[d] - 1) / g.T[d];
    g.E[d] = g.T[d] + w - 1;
    g.dscale[d] = 2.0 * p->M[d] / w;
    g.dscalef[d] = (float)g.dscale[d];
    p->ntiles *= g.nt[d];
  }
  g.vec4 = (!p->fp64 && g.T[2] % 4 == 0 && p->M[2] % 4 == 0 && (g.E[2] + 3) / 4 * 4 <= g.E3p) ? 1 : 0;
  {
    const int v = p->fp64 ? 2 : (p->bf16 ? 8 : 4);  // elements per 16 bytes
    g.gvec = (g.T[2] % v == 0 && p->M[2] % v == 0) ? 1 : 0;
    g.E2g = (g.E[2] + v - 1) / v;
  }
  auto magic = [](unsigned int d) {
    return (unsigned int)((((unsigned long long)1 << 32) + d - 1) / d);
  };
  g.div_E1 = magic((unsigned)g.E[1]);
  g.div_E2v = magic((unsigned)((g.E[2] + 3) / 4));
  g.div_E2g = magic((unsigned)g.E2g);
  for (int d = 0; d < 3; ++d) g.div_T[d] = magic((unsigned)g.T[d]);
  g.deg = p->deg;
  // psi_0 is even and largest at 0 on [-1, 1]; the margin covers the polynomial fit
  g.wmax3 = (float)std::pow(p->pswf.psi_at_0 * (1.0 + 1e-6), 3.0);
  return ESP_OK;
}

int fill_result(esp_plan_t p, const double* acc, esp_result* out) {
  if (!out) return ESP_OK;
  std::memset(out, 0, sizeof *out);
  out->energy_recip = acc[0];
  const double W[9] = {acc[1], acc[4], acc[5], acc[4], acc[2], acc[6], acc[5], acc[6], acc[3]};
  for (int i = 0; i < 9; ++i) {
    out->virial_recip[i] = W[i];
    out->pressure_recip[i] = W[i] / p->V;
  }
  out->qsum = acc[7];
  out->q2sum = acc[8];
  out->energy_self = -p->selfc * acc[8];
  out->energy_bg = -2.0 * M_PI * acc[7] * acc[7] / p->V * p->Xbg;
  out->pressure_bg = out->energy_bg / p->V;
  out->volume = p->V;
  return ESP_OK;
}

// Stage boundaries for esp_profile: event i is recorded before stage i, event i+1 after.
enum Stage { kPrep, kBin, kScan, kScatter, kZero, kSpread, kFftFwd, kScale, kFftInv, kGather, kNStage };

inline void mark(esp_plan_t p, int i) {
  if (p->profiling) {
    // "external" records stay timing events when the step is captured in a graph
    cudaEventRecordWithFlags(p->ev[i], p->stream, cudaEventRecordExternal);
    p->ev_used[i] = true;
  }
}

// The potential grid the inverse transform writes and the gather reads.
void* phi_grid(esp_plan_t p) { return p->bf16 ? p->d_phi16 : p->d_grid; }

// Forward plane transforms: the grid into d_pbox (the box of the sphere, or the full half
// spectrum through cuFFT).
int planes_forward(esp_plan_t p) {
  if (p->box_mode) {
    ESP_CUDA(p, esp::launch_fplane(p->fp64, p->pg, p->d_grid, p->d_pbox, p->d_ptw, p->stream));
    return ESP_OK;
  }
  if (p->fp64)
    ESP_CUFFT(p, cufftExecD2Z(p->fwd, (cufftDoubleReal*)p->d_grid, (cufftDoubleComplex*)p->d_pbox));
  else
    ESP_CUFFT(p, cufftExecR2C(p->fwd, (cufftReal*)p->d_grid, (cufftComplex*)p->d_pbox));
  return ESP_OK;
}

// Inverse plane transforms: the scaled columns of d_spec2 into the grid (the potential).
int planes_inverse(esp_plan_t p) {
  if (p->box_mode) {
    ESP_CUDA(p, esp::launch_iplane(p->fp64, p->bf16, p->pg, p->d_spec2, p->d_xcol, phi_grid(p), p->d_ptw,
                                   p->stream));
    return ESP_OK;
  }
  if (p->fp64)
    ESP_CUFFT(p, cufftExecZ2D(p->inv, (cufftDoubleComplex*)p->d_spec2, (cufftDoubleReal*)p->d_grid));
  else
    ESP_CUFFT(p, cufftExecC2R(p->inv, (cufftComplex*)p->d_spec2, (cufftReal*)p->d_grid));
  return ESP_OK;
}

// The full half spectrum of the real grid's current content into d_spec (cuFFT 3D R2C).
int full_spectrum(esp_plan_t p) {
  if (p->fp64)
    ESP_CUFFT(p, cufftExecD2Z(p->fwd3, (cufftDoubleReal*)p->d_grid, (cufftDoubleComplex*)p->d_spec));
  else
    ESP_CUFFT(p, cufftExecR2C(p->fwd3, (cufftReal*)p->d_grid, (cufftComplex*)p->d_spec));
  return ESP_OK;
}

int run_step(esp_plan_t p, const void* pos, const void* q, void* forces, double* acc) {
  cudaStream_t st = p->stream;
  const bool fp64 = p->fp64;
  const size_t es = fp64 ? 8 : 4;
  const size_t Mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  for (int i = 0; i <= kNStage; ++i) p->ev_used[i] = false;
  mark(p, kPrep);
  // the binning counters and control words are zero here: set at plan time, re-zeroed by
  // the spread and gather kernels of every step.  acc[0..6] is written by the sums of the
  // scaling, acc[7..9] by the sums of the binning partials.
  const bool want_f = forces != nullptr;
  const bool clear = want_f && !p->box_mode;
  if (clear) {
    // cuFFT's inverse reads the whole half spectrum: its buffer is cleared on the side
    // branch while the atoms are binned and spread (k_xfft writes only the columns that
    // meet the sphere; the library's inverse plane kernel reads the others as zero)
    ESP_CUDA(p, cudaEventRecord(p->ev_start, st));
    ESP_CUDA(p, cudaStreamWaitEvent(p->side, p->ev_start, 0));
    ESP_CUDA(p, cudaMemsetAsync(p->d_spec2, 0, 2 * es * (size_t)p->M[0] * p->M[1] * p->H2, p->side));
    ESP_CUDA(p, cudaEventRecord(p->ev_zero, p->side));
  }
  mark(p, kBin);
  ESP_CUDA(p, esp::launch_bin(p->io_double, fp64, pos, q, p->n, p->tg, p->bins, p->d_binpart,
                              p->d_grid, es * Mtot, st));
  mark(p, kSpread);
  ESP_CUDA(p, esp::launch_spread(fp64, p->tg, p->ntiles, p->spread_blocks, p->bins, p->d_wtab,
                                 p->d_grid, st));
  mark(p, kFftFwd);
  int rc;
  if ((rc = planes_forward(p)) != ESP_OK) return rc;
  mark(p, kScale);
  if (clear) ESP_CUDA(p, cudaStreamWaitEvent(st, p->ev_zero, 0));
  ESP_CUDA(p, esp::launch_xfft(fp64, true, want_f, p->xg, p->sg, p->d_pbox, p->d_spec2, p->d_xtw,
                               p->d_invw2, p->d_radtab, p->d_partials, p->d_xorder, p->d_xcol,
                               p->xactive, st));
  // the energy and virial sums finish on the side branch while the forces go on
  ESP_CUDA(p, cudaEventRecord(p->ev_fork, st));
  ESP_CUDA(p, cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  ESP_CUDA(p, esp::launch_xsum(fp64, p->d_partials, p->xactive, p->d_binpart,
                               p->n > 0 ? p->bin_blocks : 0, acc, p->side));
  ESP_CUDA(p, cudaEventRecord(p->ev_join, p->side));
  mark(p, kFftInv);
  if (want_f) {
    if ((rc = planes_inverse(p)) != ESP_OK) return rc;
    mark(p, kGather);
    ESP_CUDA(p, esp::launch_gather(fp64, p->io_double, p->bf16, p->gg, p->ntiles, p->gather_blocks,
                                   p->bins, p->d_wtab, phi_grid(p), forces, st));
  }
  ESP_CUDA(p, cudaStreamWaitEvent(st, p->ev_join, 0));
  mark(p, kNStage);
  p->spectrum_kept = !want_f;
  return ESP_OK;
}

void drop_graph(esp_plan_t p) {
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  p->graph_exec = nullptr;
}

// esp_step through a CUDA graph: the launch sequence of run_step is captured once per
// argument set (the kernels take the cell constants by value, so esp_set_cell drops the
// graph) and replayed with one launch.  The legacy default stream cannot be captured;
// there, and if capture fails, the kernels launch one by one.
int run_step_graph(esp_plan_t p, const void* pos, const void* q, void* forces, double* acc) {
  if (!p->use_graph || p->stream == nullptr) return run_step(p, pos, q, forces, acc);
  if (!(p->graph_exec && p->g_pos == pos && p->g_q == q && p->g_f == forces && p->g_acc == acc &&
        p->g_prof == p->profiling)) {
    drop_graph(p);
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(p->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return run_step(p, pos, q, forces, acc);  // the caller is capturing: just enqueue
    if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return run_step(p, pos, q, forces, acc);
    }
    const int rc = run_step(p, pos, q, forces, acc);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(p->stream, &graph);
    if (rc != ESP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess || !graph) {
      cudaGetLastError();
      p->use_graph = false;
      return run_step(p, pos, q, forces, acc);
    }
    const cudaError_t ei = cudaGraphInstantiate(&p->graph_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
      cudaGetLastError();
      p->graph_exec = nullptr;
      p->use_graph = false;
      return run_step(p, pos, q, forces, acc);
    }
    p->g_pos = pos;
    p->g_q = q;
    p->g_f = forces;
    p->g_acc = acc;
    p->g_prof = p->profiling;
  }
  ESP_CUDA(p, cudaGraphLaunch(p->graph_exec, p->stream));
  p->spectrum_kept = forces == nullptr;
  return ESP_OK;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" {

int esp_plan(esp_plan_t* out, const double cell[9], int64_t n, const int grid[3], int w,
             double c, double alpha, int precision, void* stream) {
  if (!out) return fail(nullptr, ESP_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!grid) return fail(nullptr, ESP_ERR_ARG, "grid is NULL");
  if (n < 0 || n > (int64_t)0x3fffffff) return fail(nullptr, ESP_ERR_ARG, "n out of range");
  if (w < esp::kMinP || w > esp::kMaxP)
    return fail(nullptr, ESP_ERR_ARG, "stencil width w must be in [3, 12]");
  if (!(c > 0.0) || !std::isfinite(c)) return fail(nullptr, ESP_ERR_ARG, "c must be positive");
  if (!(alpha > 0.0) || !std::isfinite(alpha))
    return fail(nullptr, ESP_ERR_ARG, "alpha (= r_c) must be positive");
  const int base = precision & 0xf;
  if (base != ESP_FP64 && base != ESP_FP32) return fail(nullptr, ESP_ERR_ARG, "bad precision");
  if ((precision & ESP_BF16_GRID) && (base != ESP_FP32 || grid[2] % 8 != 0))
    return fail(nullptr, ESP_ERR_ARG, "ESP_BF16_GRID needs ESP_FP32 and M3 a multiple of 8");
  for (int d = 0; d < 3; ++d) {
    if (grid[d] < 2 || grid[d] > 4096) return fail(nullptr, ESP_ERR_ARG, "grid size out of range");
    if (w >= grid[d]) return fail(nullptr, ESP_ERR_SUPPORT, "stencil width must be below every M_d");
  }
  if ((int64_t)grid[0] * grid[1] * grid[2] > ((int64_t)1 << 31))
    return fail(nullptr, ESP_ERR_ARG, "grid too large");

  esp_plan_t p = new esp_plan_s();
  p->fp64 = (base == ESP_FP64);
  p->io_double = p->fp64 || (precision & ESP_IO_F64);
  p->bf16 = !p->fp64 && (precision & ESP_BF16_GRID);
  p->n = n;
  for (int d = 0; d < 3; ++d) p->M[d] = grid[d];
  p->H2 = grid[2] / 2 + 1;
  p->P = w;
  p->c = c;
  p->rc = alpha;
  p->stream = (cudaStream_t)stream;
  int rc;
  auto bail = [&](int code) {
    g_plan_error = p->err;
    release(p);
    return code;
  };
  if ((rc = set_cell_matrix(p, cell, p->h, p->hinv, &p->V)) != ESP_OK) return bail(rc);
  if ((rc = check_grid(p, p->h, p->M, c, alpha, p->sg.mmax)) != ESP_OK) return bail(rc);
  if (!p->pswf.solve(c)) return bail(fail(p, ESP_ERR_ARG, "PSWF eigen-solve failed"));
  const esp::Prolate& pr = p->pswf;
  p->A = 4.0 * M_PI / pr.psi_at_0;  // 2 pi lambda_0 / C_0 with lambda_0 psi_0(0) = 2 C_0
  p->selfc = pr.psi_at_0 / (2.0 * pr.C0 * alpha);
  {
    std::vector<double> x, wq;
    esp::gauss_legendre(96, x, wq);
    double s = 0.0;
    for (size_t i = 0; i < x.size(); ++i) {
      const double u = 0.5 * (x[i] + 1.0);
      s += 0.5 * wq[i] * u * u * pr.eval(u);
    }
    p->Xbg = alpha * alpha / (2.0 * pr.C0) * s;
  }
  std::vector<double> wtab, rtab, invw2;
  if ((rc = build_window_tables(p, wtab)) != ESP_OK) return bail(rc);
  if ((rc = build_radial_tables(p, rtab)) != ESP_OK) return bail(rc);
  build_invw2(p, invw2);

  int sms = 152;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  }
  p->sms = sms;
  if ((rc = setup_tile_geom(p)) != ESP_OK) return bail(rc);
  esp::TileGeom& g = p->tg;

  esp::ScaleGeom& s = p->sg;
  for (int d = 0; d < 3; ++d) s.M[d] = p->M[d];
  s.H2 = p->H2;
  s.rdeg = p->rdeg;
  s.K2 = (c / alpha) * (c / alpha);
  s.x_per_k = alpha / c;
  s.A = p->A;
  s.K2f = (float)s.K2;
  s.x_per_kf = (float)s.x_per_k;
  s.Af = (float)s.A;
  update_cell_constants(p);

  int dev = 0;
  cudaGetDevice(&dev);
  p->device = dev;
  // the transform along axis 0: radices 8, 4, 2, 3, 5, 7, then the other prime factors;
  // 2^lognc columns per CTA, as many as keep two CTAs' shared memory within an SM
  {
    esp::XGeom& x = p->xg;
    x.M0 = p->M[0];
    x.nb1 = p->M[1];  // the full layout until the plane transforms are set up
    x.nb2 = p->H2;
    x.ncol = p->M[1] * p->H2;
    if (!radix_plan(x.M0, x.radix, x.ns_magic, &x.npass))
      return bail(fail(p, ESP_ERR_ARG, "grid size M1 has too many prime factors"));
    if (x.M0 >= (1 << 16)) return bail(fail(p, ESP_ERR_ARG, "grid size M1 too large"));
    x.lognc = 3;
    while (x.lognc > 0 && esp::xfft_smem_bytes(p->fp64, x.M0, x.lognc, p->rdeg) > 100 * 1024)
      --x.lognc;
    if (esp::xfft_smem_bytes(p->fp64, x.M0, x.lognc, p->rdeg) > 227 * 1024)
      return bail(fail(p, ESP_ERR_ARG, "grid size M1 too large for the transform along axis 1"));
    p->xblocks = esp::xfft_blocks(x);
  }

  const size_t es = p->fp64 ? 8 : 4;
  const size_t io_es = p->io_double ? 8 : 4;
  const size_t Mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  const size_t nspec = (size_t)p->M[0] * p->M[1] * p->H2;
  const size_t nn = std::max<int64_t>(n, 1);
  if ((rc = upload(p, &p->d_wtab, wtab)) != ESP_OK) return bail(rc);
  if ((rc = upload(p, &p->d_radtab, rtab)) != ESP_OK) return bail(rc);
  if ((rc = upload(p, &p->d_invw2, invw2)) != ESP_OK) return bail(rc);
#define ALLOC(ptr, bytes)                                                    \
  do {                                                                       \
    cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                    \
    if (e_ != cudaSuccess) return bail(cuda_fail(p, e_, "cudaMalloc " #ptr)); \
  } while (0)
  ALLOC(p->d_grid, es * Mtot);
  ALLOC(p->d_spec, 2 * es * nspec);
  ALLOC(p->d_spec2, 2 * es * nspec);
  ALLOC(p->d_pbox, 2 * es * nspec);
  ALLOC(p->d_ptw, 2 * es * (size_t)(p->M[1] + p->M[2]));
  if (p->bf16) ALLOC(p->d_phi16, 2 * Mtot);
  p->bin_blocks = esp::bin_blocks(n);
  {
    esp::Bins& b = p->bins;
    b.cap = esp::bin_capacity(n, p->ntiles);
    const size_t nslot = (size_t)p->ntiles * b.cap;
    ALLOC(b.count, sizeof(int) * (size_t)p->ntiles);
    ALLOC(b.tcount, sizeof(int) * (size_t)p->ntiles);
    ALLOC(b.tq, 4 * es * nslot);
    ALLOC(b.lb, sizeof(int) * nslot);
    ALLOC(b.idx, sizeof(int) * nslot);
    ALLOC(b.otq, 4 * es * nn);
    ALLOC(b.ob, 3 * sizeof(int) * nn);
    ALLOC(b.oidx, sizeof(int) * nn);
    ALLOC(b.ctrl, sizeof(int) * esp::kCtrl);
    ALLOC(b.hq, sizeof(float) * esp::kHQ * (size_t)p->ntiles);
  }
  ALLOC(p->d_binpart, sizeof(double) * 3 * p->bin_blocks);
  ALLOC(p->d_accum, sizeof(double) * ESP_ACCUM_LEN);
  ALLOC(p->d_partials, sizeof(double) * 7 * (size_t)p->xblocks);
  ALLOC(p->d_xtw, 2 * es * (size_t)p->M[0]);
  ALLOC(p->d_xorder, sizeof(int) * (size_t)p->xblocks);
  ALLOC(p->d_xcol, (size_t)p->xg.ncol);
#undef ALLOC
  (void)io_es;
  {
    cudaError_t e = cudaMemset(p->bins.count, 0, sizeof(int) * (size_t)p->ntiles);
    if (e == cudaSuccess) e = cudaMemset(p->bins.tcount, 0, sizeof(int) * (size_t)p->ntiles);
    if (e == cudaSuccess) e = cudaMemset(p->bins.ctrl, 0, sizeof(int) * esp::kCtrl);
    if (e == cudaSuccess) e = cudaMemset(p->bins.hq, 0, sizeof(float) * esp::kHQ * (size_t)p->ntiles);
    if (e == cudaSuccess) e = cudaMemset(p->d_accum, 0, sizeof(double) * ESP_ACCUM_LEN);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_accum, sizeof(double) * ESP_ACCUM_LEN);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_xorder, sizeof(int) * (size_t)p->xblocks);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&p->h_xcol, (size_t)p->xg.ncol);
    if (e != cudaSuccess) return bail(cuda_fail(p, e, "plan workspace set-up"));
  }
  {
    // roots of unity for the transform along axis 0, FP64 on the host
    std::vector<double> tw(2 * (size_t)p->M[0]);
    for (int m = 0; m < p->M[0]; ++m) {
      tw[2 * m] = std::cos(2.0 * M_PI * m / p->M[0]);
      tw[2 * m + 1] = -std::sin(2.0 * M_PI * m / p->M[0]);
    }
    // and the M1 then M2 roots of the plane transforms
    std::vector<double> ptw;
    for (int d = 1; d <= 2; ++d)
      for (int m = 0; m < p->M[d]; ++m) {
        ptw.push_back(std::cos(2.0 * M_PI * m / p->M[d]));
        ptw.push_back(-std::sin(2.0 * M_PI * m / p->M[d]));
      }
    cudaError_t e;
    if (p->fp64) {
      e = cudaMemcpy(p->d_xtw, tw.data(), sizeof(double) * tw.size(), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(p->d_ptw, ptw.data(), sizeof(double) * ptw.size(), cudaMemcpyHostToDevice);
    } else {
      std::vector<float> twf(tw.begin(), tw.end());
      e = cudaMemcpy(p->d_xtw, twf.data(), sizeof(float) * twf.size(), cudaMemcpyHostToDevice);
      std::vector<float> ptwf(ptw.begin(), ptw.end());
      if (e == cudaSuccess)
        e = cudaMemcpy(p->d_ptw, ptwf.data(), sizeof(float) * ptwf.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess)
      e = esp::configure_xfft(p->fp64, esp::xfft_smem_bytes(p->fp64, p->xg.M0, p->xg.lognc, p->rdeg));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_zero, cudaEventDisableTiming);
    if (e != cudaSuccess) return bail(cuda_fail(p, e, "transform set-up"));
    if ((rc = setup_planes(p)) != ESP_OK) return bail(rc);
    if ((rc = update_xfft_tasks(p)) != ESP_OK) return bail(rc);
  }
  {
    // plane transforms: every i0 plane over (i1, i2), batched
    int n2[2] = {p->M[1], p->M[2]};
    const int nr = p->M[1] * p->M[2], nc = p->M[1] * p->H2;
    cufftResult r1 = cufftPlanMany(&p->fwd, 2, n2, nullptr, 1, nr, nullptr, 1, nc,
                                   p->fp64 ? CUFFT_D2Z : CUFFT_R2C, p->M[0]);
    if (r1 != CUFFT_SUCCESS) return bail(fail(p, ESP_ERR_CUFFT, "cufftPlanMany (forward) failed"));
    p->have_fwd = true;
    cufftResult r2 = cufftPlanMany(&p->inv, 2, n2, nullptr, 1, nc, nullptr, 1, nr,
                                   p->fp64 ? CUFFT_Z2D : CUFFT_C2R, p->M[0]);
    if (r2 != CUFFT_SUCCESS) return bail(fail(p, ESP_ERR_CUFFT, "cufftPlanMany (inverse) failed"));
    p->have_inv = true;
    cufftResult r3 = cufftPlan3d(&p->fwd3, p->M[0], p->M[1], p->M[2], p->fp64 ? CUFFT_D2Z : CUFFT_R2C);
    if (r3 != CUFFT_SUCCESS) return bail(fail(p, ESP_ERR_CUFFT, "cufftPlan3d (forward) failed"));
    p->have_fwd3 = true;
    if (cufftSetStream(p->fwd, p->stream) != CUFFT_SUCCESS ||
        cufftSetStream(p->inv, p->stream) != CUFFT_SUCCESS ||
        cufftSetStream(p->fwd3, p->stream) != CUFFT_SUCCESS)
      return bail(fail(p, ESP_ERR_CUFFT, "cufftSetStream failed"));
  }
  {
    const size_t ss = esp::spread_smem_bytes(p->fp64, g),
                 gs = esp::gather_smem_bytes(p->fp64, g, p->bf16);
    if (ss > 227 * 1024 || gs > 227 * 1024)
      return bail(fail(p, ESP_ERR_ARG, "tile does not fit in shared memory"));
    cudaError_t e = esp::configure_kernels(p->fp64, w, ss, gs, p->bf16);
    if (e != cudaSuccess) return bail(cuda_fail(p, e, "cudaFuncSetAttribute"));
    int occ_s = 1, occ_g = 1;
    e = esp::occupancy(p->fp64, p->io_double, w, ss, gs, &occ_s, &occ_g, p->bf16);
    if (e != cudaSuccess) return bail(cuda_fail(p, e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor"));
    p->spread_blocks = std::max(1, std::min(p->ntiles, sms * std::max(occ_s, 1)));
    p->gather_blocks = std::max(1, std::min(p->ntiles, sms * std::max(occ_g, 1)));
  }
  *out = p;
  return ESP_OK;
}

int esp_set_cell(esp_plan_t p, const double cell[9]) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  double h[9], hinv[9], V;
  int rc;
  if ((rc = set_cell_matrix(p, cell, h, hinv, &V)) != ESP_OK) return rc;
  int mmax[3];
  if ((rc = check_grid(p, h, p->M, p->c, p->rc, mmax)) != ESP_OK) return rc;
  std::memcpy(p->h, h, sizeof h);
  std::memcpy(p->hinv, hinv, sizeof hinv);
  p->V = V;
  for (int d = 0; d < 3; ++d) p->sg.mmax[d] = mmax[d];
  update_cell_constants(p);
  p->spectrum_kept = false;
  drop_graph(p);
  if ((rc = setup_planes(p)) != ESP_OK) return rc;
  return update_xfft_tasks(p);
}

int esp_set_stream(esp_plan_t p, void* stream) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  p->stream = (cudaStream_t)stream;
  drop_graph(p);
  if (cufftSetStream(p->fwd, p->stream) != CUFFT_SUCCESS ||
      cufftSetStream(p->inv, p->stream) != CUFFT_SUCCESS ||
      cufftSetStream(p->fwd3, p->stream) != CUFFT_SUCCESS)
    return fail(p, ESP_ERR_CUFFT, "cufftSetStream failed");
  return ESP_OK;
}

int esp_step(esp_plan_t p, const void* pos, const void* q, void* forces, double* d_accum) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q)) return fail(p, ESP_ERR_ARG, "pos or q is NULL");
  DeviceGuard guard(p->device);
  return run_step_graph(p, pos, q, forces, d_accum ? d_accum : p->d_accum);
}

int esp_energy_pressure(esp_plan_t p, const void* pos, const void* q, esp_result* out) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (!out) return fail(p, ESP_ERR_ARG, "out is NULL");
  if (p->n > 0 && (!pos || !q)) return fail(p, ESP_ERR_ARG, "pos or q is NULL");
  DeviceGuard guard(p->device);
  int rc = run_step(p, pos, q, nullptr, p->d_accum);
  if (rc != ESP_OK) return rc;
  ESP_CUDA(p, cudaMemcpyAsync(p->h_accum, p->d_accum, sizeof(double) * ESP_ACCUM_LEN,
                              cudaMemcpyDeviceToHost, p->stream));
  ESP_CUDA(p, cudaStreamSynchronize(p->stream));
  fill_result(p, p->h_accum, out);
  if (p->h_accum[9] > 0.0) {
    p->spectrum_kept = false;
    return fail(p, ESP_ERR_NONFINITE, "non-finite position or charge");
  }
  return ESP_OK;
}

int esp_forces(esp_plan_t p, const void* pos, const void* q, void* forces) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q || !forces)) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  return run_step(p, pos, q, forces ? forces : nullptr, p->d_accum);
}

int esp_forces_from_spectrum(esp_plan_t p, void* forces) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && !forces) return fail(p, ESP_ERR_ARG, "forces is NULL");
  if (!p->spectrum_kept) return fail(p, ESP_ERR_STATE, "no spectrum kept for these positions");
  DeviceGuard guard(p->device);
  cudaStream_t st = p->stream;
  const bool fp64 = p->fp64;
  if (!p->box_mode)
    ESP_CUDA(p, cudaMemsetAsync(p->d_spec2, 0,
                                2 * (fp64 ? 8 : 4) * (size_t)p->M[0] * p->M[1] * p->H2, st));
  // the kept plane transforms take the transform along i0, the scaling and its inverse
  ESP_CUDA(p, esp::launch_xfft(fp64, true, true, p->xg, p->sg, p->d_pbox, p->d_spec2, p->d_xtw,
                               p->d_invw2, p->d_radtab, p->d_partials, p->d_xorder, p->d_xcol,
                               p->xactive, st));
  ESP_CUDA(p, esp::launch_xsum(fp64, p->d_partials, p->xactive, p->d_binpart,
                               p->n > 0 ? p->bin_blocks : 0, p->d_accum, st));
  int rc;
  if ((rc = planes_inverse(p)) != ESP_OK) return rc;
  ESP_CUDA(p, esp::launch_gather(fp64, p->io_double, p->bf16, p->gg, p->ntiles, p->gather_blocks,
                                 p->bins, p->d_wtab, phi_grid(p), forces, st));
  p->spectrum_kept = false;
  return ESP_OK;
}

// Field variants: the step without forces (the spectrum X stays), fields built from X,
// their inverse transforms (batched), and window interpolation at the atoms.
// kind 0: per-atom energy (1 field), 1: ik-differentiation forces (3), 2: per-atom virial (6).
int run_fields(esp_plan_t p, const void* pos, const void* q, int kind, void* out, double coef) {
  const int nf = kind == 0 ? 1 : (kind == 1 ? 3 : 6);
  const size_t es = p->fp64 ? 8 : 4;
  const size_t ns = (size_t)p->M[0] * p->M[1] * p->H2;
  const size_t Mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  if (!p->d_fspec) {
    ESP_CUDA(p, cudaMalloc(&p->d_fspec, 6 * ns * 2 * es));
    ESP_CUDA(p, cudaMalloc(&p->d_fgrid, 6 * Mtot * es));
  }
  auto batched = [&](cufftHandle* h, bool* have, int batch) -> int {
    if (*have) return ESP_OK;
    int n[3] = {p->M[0], p->M[1], p->M[2]};
    if (cufftPlanMany(h, 3, n, nullptr, 1, (int)ns, nullptr, 1, (int)Mtot,
                      p->fp64 ? CUFFT_Z2D : CUFFT_C2R, batch) != CUFFT_SUCCESS)
      return fail(p, ESP_ERR_CUFFT, "cufftPlanMany (field transforms) failed");
    *have = true;
    if (cufftSetStream(*h, p->stream) != CUFFT_SUCCESS)
      return fail(p, ESP_ERR_CUFFT, "cufftSetStream failed");
    return ESP_OK;
  };
  int rc = ESP_OK;
  if (nf == 1 && (rc = batched(&p->inv3, &p->have_inv3, 1)) != ESP_OK) return rc;
  if (nf == 3 && (rc = batched(&p->finv3, &p->have_finv3, 3)) != ESP_OK) return rc;
  if (nf == 6 && (rc = batched(&p->finv6, &p->have_finv6, 6)) != ESP_OK) return rc;
  const cufftHandle plan = nf == 1 ? p->inv3 : (nf == 3 ? p->finv3 : p->finv6);
  if (cufftSetStream(plan, p->stream) != CUFFT_SUCCESS)
    return fail(p, ESP_ERR_CUFFT, "cufftSetStream failed");
  if ((rc = run_step(p, pos, q, nullptr, p->d_accum)) != ESP_OK) return rc;
  cudaStream_t st = p->stream;
  // the full 3D half spectrum of the spread grid (the step keeps only the box of the sphere)
  if ((rc = full_spectrum(p)) != ESP_OK) return rc;
  ESP_CUDA(p, esp::launch_fields(p->fp64, kind, p->sg, p->d_spec, p->d_invw2, p->d_radtab,
                                 p->d_fspec, st));
  if (p->fp64)
    ESP_CUFFT(p, cufftExecZ2D(plan, (cufftDoubleComplex*)p->d_fspec, (cufftDoubleReal*)p->d_fgrid));
  else
    ESP_CUFFT(p, cufftExecC2R(plan, (cufftComplex*)p->d_fspec, (cufftReal*)p->d_fgrid));
  // gathers of up to 3 fields at a time (one at a time when 3 tiles do not fit)
  const int per = esp::fields_smem_bytes(p->fp64, p->P, 3) <= 227 * 1024 ? 3 : 1;
  for (int f0 = 0; f0 < nf; f0 += per) {
    const int k = std::min(per, nf - f0);
    ESP_CUDA(p, esp::launch_gather_fields(p->fp64, p->io_double, p->tg, p->ntiles, p->gather_blocks, k,
                                          p->bins, p->d_wtab,
                                          (const unsigned char*)p->d_fgrid + (size_t)f0 * Mtot * es,
                                          (int64_t)Mtot, coef, out, nf, f0, st));
  }
  p->spectrum_kept = true;
  return ESP_OK;
}

int esp_forces_ik(esp_plan_t p, const void* pos, const void* q, void* forces) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q || !forces)) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  return run_fields(p, pos, q, 1, forces, -p->gg.fscale);
}

int esp_local_virial(esp_plan_t p, const void* pos, const void* q, void* virial) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q || !virial)) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  return run_fields(p, pos, q, 2, virial, 0.5 * p->gg.fscale);
}

int esp_atom_energy(esp_plan_t p, const void* pos, const void* q, void* energy) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q || !energy)) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  return run_fields(p, pos, q, 0, energy, 0.5 * p->gg.fscale);
}

int esp_near(esp_plan_t p, const void* pos, const void* q, void* forces, int add,
             double* d_out) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (!d_out || (p->n > 0 && (!pos || !q || !forces)))
    return fail(p, ESP_ERR_ARG, "pos, q, forces or d_out is NULL");
  DeviceGuard guard(p->device);
  // cell list of the current cell: nc bins of at least r_c / 2 per axis, R neighbours each
  // side, blocks of up to 2 x 2 x 2 bins per CTA
  esp::NearGeom& ng = p->ng;
  int ncells = 1;
  for (int d = 0; d < 3; ++d) {
    // perpendicular width of the cell along reduced axis d: 1 / |row d of h^{-1}|
    const double* r = p->hinv + 3 * d;
    const double width = 1.0 / std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    ng.nc[d] = std::max(1, (int)std::min(1024.0, std::floor(2.0 * width / p->rc)));
    ng.R[d] = std::max(1, (int)std::ceil(p->rc * ng.nc[d] / width));
    ng.B[d] = std::min(2, ng.nc[d]);
    ng.nb[d] = (ng.nc[d] + ng.B[d] - 1) / ng.B[d];
    ng.inv_nc[d] = 1.0 / ng.nc[d];
    ncells *= ng.nc[d];
  }
  if (esp::near_region_cells(ng) > esp::kNearMaxRegion ||
      esp::near_pairs_smem(p->fp64, ng) > esp::kNearMaxSmem)
    return fail(p, ESP_ERR_SUPPORT, "cell too narrow for the near-part cell list (a block's "
                                    "neighbourhood exceeds 2048 cells or the shared memory of "
                                    "the pair kernel): r_c is many cell widths");
  for (int i = 0; i < 9; ++i) {
    ng.h[i] = p->h[i];
    ng.hinv[i] = p->hinv[i];
  }
  ng.rc = p->rc;
  ng.inv_rc = 1.0 / p->rc;
  if (!p->d_neartab) {
    std::vector<double> tab;
    int rc = build_near_tables(p, tab);
    if (rc != ESP_OK) return rc;
    if ((rc = upload(p, &p->d_neartab, tab)) != ESP_OK) return rc;
    const size_t es = p->fp64 ? 8 : 4;
    const size_t nn = std::max<int64_t>(p->n, 1);
    ESP_CUDA(p, cudaMalloc(&p->d_ncell, nn * sizeof(int)));
    ESP_CUDA(p, cudaMalloc(&p->d_nrank, nn * sizeof(int)));
    ESP_CUDA(p, cudaMalloc(&p->d_nidx, nn * sizeof(int)));
    ESP_CUDA(p, cudaMalloc(&p->d_nxq_tmp, nn * 4 * es));
    ESP_CUDA(p, cudaMalloc(&p->d_nxq, nn * 4 * es));
    ESP_CUDA(p, cudaMalloc(&p->d_noff, (size_t)esp::kNearMaxRegion * 4 * es));
  }
  ng.ndeg = p->near_ndeg;
  if (ncells > p->near_cells_alloc) {
    if (p->d_ncount) cudaFree(p->d_ncount);
    if (p->d_ncoff) cudaFree(p->d_ncoff);
    p->d_ncount = nullptr;
    p->d_ncoff = nullptr;
    p->near_cells_alloc = 0;
    ESP_CUDA(p, cudaMalloc(&p->d_ncount, (size_t)ncells * sizeof(int)));
    ESP_CUDA(p, cudaMalloc(&p->d_ncoff, ((size_t)ncells + 1) * sizeof(int)));
    ESP_CUDA(p, cudaMemset(p->d_ncount, 0, (size_t)ncells * sizeof(int)));
    p->near_cells_alloc = ncells;
  }
  cudaStream_t st = p->stream;
  ESP_CUDA(p, esp::launch_near_bin(p->io_double, p->fp64, pos, q, p->n, ng, p->d_ncount,
                                   p->d_ncell, p->d_nrank, p->d_nxq_tmp, st));
  ESP_CUDA(p, esp::launch_near_scan(p->d_ncount, p->d_ncoff, ncells, st));
  ESP_CUDA(p, esp::launch_near_scatter(p->fp64, p->n, p->d_ncell, p->d_nrank, p->d_ncoff,
                                       p->d_nxq_tmp, p->d_nxq, p->d_nidx, st));
  ESP_CUDA(p, esp::launch_near_pairs(p->fp64, p->io_double, ng, ncells, p->d_ncoff, p->d_nxq,
                                     p->d_nidx, p->d_neartab, p->d_noff, p->d_nxq_tmp, forces,
                                     add, p->n, d_out, st));
  return ESP_OK;
}

int esp_cell_gradient(esp_plan_t p, const void* pos, const void* forces, const double* d_accum,
                      double* d_grad) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (!d_grad || (p->n > 0 && (!pos || !forces)))
    return fail(p, ESP_ERR_ARG, "pos, forces or d_grad is NULL");
  DeviceGuard guard(p->device);
  esp::CellGradArgs c;
  for (int i = 0; i < 9; ++i) c.hinv[i] = p->hinv[i];
  c.bg_coef = -2.0 * M_PI / p->V * p->Xbg;
  ESP_CUDA(p, esp::launch_cell_grad(p->io_double, pos, forces, p->n, c,
                                    d_accum ? d_accum : p->d_accum, d_grad, p->stream));
  return ESP_OK;
}

namespace {
// The device address of page-locked (pinned or registered) host memory, else NULL.
const void* mapped_host(const void* ptr) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}
}  // namespace

int esp_compute_host(esp_plan_t p, const void* pos, const void* q, void* forces,
                     esp_result* out) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (p->n > 0 && (!pos || !q)) return fail(p, ESP_ERR_ARG, "pos or q is NULL");
  DeviceGuard guard(p->device);
  const size_t io_es = p->io_double ? 8 : 4;
  const size_t nn = (size_t)std::max<int64_t>(p->n, 1);
  if (!p->d_io_pos) {
    ESP_CUDA(p, cudaMalloc(&p->d_io_pos, 3 * io_es * nn));
    ESP_CUDA(p, cudaMalloc(&p->d_io_q, io_es * nn));
    ESP_CUDA(p, cudaMalloc(&p->d_io_f, 3 * io_es * nn));
  }
  cudaStream_t st = p->stream;
  // Page-locked host inputs are read by the binning kernel in place (through their device
  // mapping); other host memory is copied to the plan's staging buffers first.
  const void* dpos = p->d_io_pos;
  const void* dq = p->d_io_q;
  if (p->n > 0) {
    const void* mpos = mapped_host(pos);
    const void* mq = mapped_host(q);
    if (mpos && mq) {
      dpos = mpos;
      dq = mq;
    } else {
      ESP_CUDA(p, cudaMemcpyAsync(p->d_io_pos, pos, 3 * io_es * p->n, cudaMemcpyHostToDevice, st));
      ESP_CUDA(p, cudaMemcpyAsync(p->d_io_q, q, io_es * p->n, cudaMemcpyHostToDevice, st));
    }
  }
  // the step through the captured graph: one capture serves every call with the same
  // input buffers (plain launches on the legacy default stream)
  int rc = run_step_graph(p, dpos, dq, forces ? p->d_io_f : nullptr, p->d_accum);
  if (rc != ESP_OK) return rc;
  // Results back: into page-locked, 16-byte aligned host forces a kernel writes through
  // the device mapping with coalesced 16-byte stores (faster over the CPU-GPU link than a
  // copy-engine transfer of this size); otherwise two copies.
  void* fmap = (forces && p->n > 0) ? const_cast<void*>(mapped_host(forces)) : nullptr;
  void* amap = const_cast<void*>(mapped_host(p->h_accum));
  const size_t fbytes = 3 * io_es * (size_t)p->n;
  if (fmap && amap && ((uintptr_t)fmap & 15) == 0) {
    ESP_CUDA(p, esp::launch_copy_out(p->d_io_f, fmap, (int64_t)(fbytes / 4), p->d_accum,
                                     (double*)amap, ESP_ACCUM_LEN, p->sms, st));
  } else {
    ESP_CUDA(p, cudaMemcpyAsync(p->h_accum, p->d_accum, sizeof(double) * ESP_ACCUM_LEN,
                                cudaMemcpyDeviceToHost, st));
    if (forces && p->n > 0)
      ESP_CUDA(p, cudaMemcpyAsync(forces, p->d_io_f, fbytes, cudaMemcpyDeviceToHost, st));
  }
  ESP_CUDA(p, cudaStreamSynchronize(st));
  fill_result(p, p->h_accum, out);
  if (p->h_accum[9] > 0.0) return fail(p, ESP_ERR_NONFINITE, "non-finite position or charge");
  return ESP_OK;
}

int esp_result_from_accum(esp_plan_t p, const double accum_host[ESP_ACCUM_LEN],
                          esp_result* out) {
  if (!p || !accum_host || !out) return fail(p, ESP_ERR_ARG, "NULL argument");
  return fill_result(p, accum_host, out);
}

int esp_copy_grid(esp_plan_t p, void* host_dst) {
  if (!p || !host_dst) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  const size_t es = p->fp64 ? 8 : 4;
  const size_t Mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  ESP_CUDA(p, cudaStreamSynchronize(p->stream));
  ESP_CUDA(p, cudaMemcpy(host_dst, p->d_grid, es * Mtot, cudaMemcpyDeviceToHost));
  return ESP_OK;
}

int esp_copy_spectrum(esp_plan_t p, void* host_dst) {
  if (!p || !host_dst) return fail(p, ESP_ERR_ARG, "NULL argument");
  DeviceGuard guard(p->device);
  const size_t es = p->fp64 ? 8 : 4;
  const size_t ns = (size_t)p->M[0] * p->M[1] * p->H2;
  int rc;
  if ((rc = full_spectrum(p)) != ESP_OK) return rc;
  ESP_CUDA(p, cudaStreamSynchronize(p->stream));
  ESP_CUDA(p, cudaMemcpy(host_dst, p->d_spec, 2 * es * ns, cudaMemcpyDeviceToHost));
  return ESP_OK;
}

int esp_plan_info(esp_plan_t p, double* info, int len) {
  if (!p || !info || len < 0) return fail(p, ESP_ERR_ARG, "NULL argument");
  const double v[18] = {p->c,
                        p->rc,
                        p->pswf.psi_at_0,
                        p->pswf.C0,
                        p->pswf.lambda0,
                        (double)p->deg,
                        (double)p->rdeg,
                        p->fit_err,
                        p->rfit_err,
                        (double)p->ntiles,
                        (double)p->tg.T[0],
                        (double)p->tg.T[1],
                        (double)p->tg.T[2],
                        p->box_mode ? 7.0 : 5.0,  // bin, spread, [k_fplane], k_xfft, k_xsum, [k_iplane], gather
                        p->Xbg,
                        p->box_mode ? 1.0 : 0.0,
                        (double)p->xg.nb1,
                        (double)p->xg.nb2};
  for (int i = 0; i < std::min(len, 18); ++i) info[i] = v[i];
  return ESP_OK;
}

int esp_profile(esp_plan_t p, int enable) {
  if (!p) return fail(nullptr, ESP_ERR_ARG, "plan is NULL");
  if (enable && !p->ev[0]) {
    DeviceGuard guard(p->device);
    for (int i = 0; i <= kNStage; ++i) ESP_CUDA(p, cudaEventCreate(&p->ev[i]));
  }
  p->profiling = enable != 0;
  return ESP_OK;
}

int esp_profile_read(esp_plan_t p, double* stage_ms, int len) {
  if (!p || !stage_ms) return fail(p, ESP_ERR_ARG, "NULL argument");
  if (!p->profiling) return fail(p, ESP_ERR_STATE, "profiling is off");
  DeviceGuard guard(p->device);
  ESP_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int i = 0; i < std::min(len, (int)kNStage); ++i) {
    stage_ms[i] = 0.0;
    int j = i + 1;  // the next recorded boundary ends stage i
    while (j <= kNStage && !p->ev_used[j]) ++j;
    if (!p->ev_used[i] || j > kNStage) continue;
    float ms = 0.f;
    ESP_CUDA(p, cudaEventElapsedTime(&ms, p->ev[i], p->ev[j]));
    stage_ms[i] = ms;
  }
  return ESP_OK;
}

int esp_destroy(esp_plan_t p) {
  release(p);
  return ESP_OK;
}

const char* esp_last_error(esp_plan_t p) {
  return p ? p->err.c_str() : g_plan_error.c_str();
}

double esp_c_from_tolerance(double delta) { return esp::c_from_tolerance(delta); }

int esp_pressure_coupling(const double P[9], int mode, double* out) {
  if (!P || !out) return fail(nullptr, ESP_ERR_ARG, "NULL argument");
  switch (mode) {
    case ESP_COUPLE_ISO:
      out[0] = (P[0] + P[4] + P[8]) / 3.0;
      return 1;
    case ESP_COUPLE_SEMI:
      out[0] = 0.5 * (P[0] + P[4]);
      out[1] = P[8];
      return 2;
    case ESP_COUPLE_ANISO:
      out[0] = P[0];
      out[1] = P[4];
      out[2] = P[8];
      return 3;
    case ESP_COUPLE_FLEXIBLE:
      out[0] = P[0];
      out[1] = P[4];
      out[2] = P[8];
      out[3] = P[1];
      out[4] = P[2];
      out[5] = P[5];
      return 6;
    default:
      return fail(nullptr, ESP_ERR_ARG, "unknown pressure coupling mode");
  }
}

}  // extern "C"

// ---- allocation-free spreading ------------------------------------------------------------
// Scratch for esp_spread_noalloc: one file-scope device array with fixed offsets.  Host
// code must not take the array's name as a device address: each device's address comes
// from cudaGetSymbolAddress, once, with that device current.
namespace {

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// slots of the binned atoms: at least 32 per tile at the largest tile count
constexpr size_t kNoAllocSlots = 2 * (size_t)ESP_NOALLOC_MAX_ATOMS > 32 * (size_t)ESP_NOALLOC_MAX_TILES
                                     ? 2 * (size_t)ESP_NOALLOC_MAX_ATOMS
                                     : 32 * (size_t)ESP_NOALLOC_MAX_TILES;

struct NoAllocLayout {
  size_t count, tcount, ctrl, hq, binpart, tq, lb, idx, otq, ob, oidx, wtab, total;
};

constexpr NoAllocLayout noalloc_layout() {
  const size_t N = ESP_NOALLOC_MAX_ATOMS, T = ESP_NOALLOC_MAX_TILES, S = kNoAllocSlots;
  const size_t nbin = (N + esp::kThreads - 1) / esp::kThreads;
  NoAllocLayout L{};
  size_t o = 0;
  L.count = o;   o = al256(o + sizeof(int) * T);
  L.tcount = o;  o = al256(o + sizeof(int) * T);
  L.ctrl = o;    o = al256(o + sizeof(int) * esp::kCtrl);
  L.hq = o;      o = al256(o + sizeof(float) * esp::kHQ * T);
  L.binpart = o; o = al256(o + 3 * 8 * nbin);
  L.tq = o;      o = al256(o + 32 * S);
  L.lb = o;      o = al256(o + sizeof(int) * S);
  L.idx = o;     o = al256(o + sizeof(int) * S);
  L.otq = o;     o = al256(o + 32 * N);
  L.ob = o;      o = al256(o + 3 * sizeof(int) * N);
  L.oidx = o;    o = al256(o + sizeof(int) * N);
  L.wtab = o;    o = al256(o + sizeof(double) * 2 * (esp::kMaxDeg + 1) * esp::kMaxP);
  L.total = o;
  return L;
}

constexpr NoAllocLayout kNoAlloc = noalloc_layout();

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAlloc.total];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned char* g_noalloc_addr[kMaxDevices] = {};

// device address of the scratch array for the current device (set up on first use)
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, ESP_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
    g_noalloc_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_noalloc_addr[dev];
  return ESP_OK;
}


// The window table reaches the scratch array as a kernel argument (by value), so no
// host buffer has to outlive the call.  At most 2 (kMaxDeg + 1) kMaxP values.
struct WindowTableArg {
  double v[2 * (esp::kMaxDeg + 1) * esp::kMaxP];
  int n;
};

__global__ void k_put_window_table(WindowTableArg t, void* dst, int fp64) {
  for (int i = threadIdx.x; i < t.n; i += blockDim.x) {
    if (fp64)
      static_cast<double*>(dst)[i] = t.v[i];
    else
      static_cast<float*>(dst)[i] = (float)t.v[i];
  }
}

// The last window table built, so that repeated calls with the same (c, P, precision)
// skip the eigen-solve and the polynomial fits.
struct NoAllocTableCache {
  bool valid = false;
  double c = 0.0;
  int P = 0;
  bool fp64 = false;
  int deg = 0;
  double psi_at_0 = 0.0;
  std::vector<double> tab;
};
std::mutex g_table_mu;
NoAllocTableCache g_table_cache;

}  // namespace

extern "C" int esp_spread_noalloc(const double cell[9], int64_t n, const int grid[3], int w,
                                  double c, int precision, const void* pos, const void* q,
                                  void* grid_out, void* stream) {
  if (!grid || !grid_out) return fail(nullptr, ESP_ERR_ARG, "grid or grid_out is NULL");
  if (n < 0 || n > ESP_NOALLOC_MAX_ATOMS)
    return fail(nullptr, ESP_ERR_ARG, "n exceeds ESP_NOALLOC_MAX_ATOMS for esp_spread_noalloc");
  if (n > 0 && (!pos || !q)) return fail(nullptr, ESP_ERR_ARG, "pos or q is NULL");
  if (w < esp::kMinP || w > esp::kMaxP)
    return fail(nullptr, ESP_ERR_ARG, "stencil width w must be in [3, 12]");
  if (!(c > 0.0) || !std::isfinite(c)) return fail(nullptr, ESP_ERR_ARG, "c must be positive");
  const int base = precision & 0xf;
  if (base != ESP_FP64 && base != ESP_FP32) return fail(nullptr, ESP_ERR_ARG, "bad precision");
  for (int d = 0; d < 3; ++d) {
    if (grid[d] < 2 || grid[d] > 4096) return fail(nullptr, ESP_ERR_ARG, "grid size out of range");
    if (w >= grid[d]) return fail(nullptr, ESP_ERR_SUPPORT, "stencil width must be below every M_d");
  }
  // host-side set-up in a plan object that owns no device memory
  esp_plan_s tmp;
  esp_plan_t p = &tmp;
  p->fp64 = (base == ESP_FP64);
  p->io_double = p->fp64 || (precision & ESP_IO_F64);
  p->n = n;
  for (int d = 0; d < 3; ++d) p->M[d] = grid[d];
  p->H2 = grid[2] / 2 + 1;
  p->P = w;
  p->c = c;
  p->stream = (cudaStream_t)stream;
  // errors after this point are reported through esp_last_error(NULL)
  auto report = [&](int code) {
    if (code != ESP_OK) g_plan_error = p->err;
    return code;
  };
  int rc;
  if ((rc = set_cell_matrix(p, cell, p->h, p->hinv, &p->V)) != ESP_OK) return report(rc);
  WindowTableArg targ;
  {
    std::lock_guard<std::mutex> lock(g_table_mu);
    NoAllocTableCache& tc = g_table_cache;
    if (!(tc.valid && tc.c == c && tc.P == w && tc.fp64 == p->fp64)) {
      tc.valid = false;
      if (!p->pswf.solve(c)) return report(fail(p, ESP_ERR_ARG, "PSWF eigen-solve failed"));
      if ((rc = build_window_tables(p, tc.tab)) != ESP_OK) return report(rc);
      tc.c = c;
      tc.P = w;
      tc.fp64 = p->fp64;
      tc.deg = p->deg;
      tc.psi_at_0 = p->pswf.psi_at_0;
      tc.valid = true;
    }
    p->deg = tc.deg;
    p->pswf.psi_at_0 = tc.psi_at_0;  // the one PSWF constant the tile set-up reads
    if (tc.tab.size() > sizeof targ.v / sizeof targ.v[0])
      return report(fail(p, ESP_ERR_ARG, "window table too large"));
    targ.n = (int)tc.tab.size();
    std::copy(tc.tab.begin(), tc.tab.end(), targ.v);
  }
  if ((rc = setup_tile_geom(p)) != ESP_OK) return report(rc);
  if (p->ntiles > ESP_NOALLOC_MAX_TILES)
    return report(fail(p, ESP_ERR_ARG, "grid exceeds ESP_NOALLOC_MAX_TILES tiles for esp_spread_noalloc"));
  esp::TileGeom& g = p->tg;
  update_cell_constants(p);

  unsigned char* S = nullptr;
  if ((rc = noalloc_scratch(&S)) != ESP_OK) return rc;  // reports through g_plan_error
  esp::Bins bins{};
  bins.cap = std::max(32, std::min(esp::bin_capacity(n, p->ntiles),
                                   (int)(kNoAllocSlots / (size_t)p->ntiles / 32 * 32)));
  bins.count = reinterpret_cast<int*>(S + kNoAlloc.count);
  bins.tcount = reinterpret_cast<int*>(S + kNoAlloc.tcount);
  bins.ctrl = reinterpret_cast<int*>(S + kNoAlloc.ctrl);
  bins.hq = reinterpret_cast<float*>(S + kNoAlloc.hq);
  bins.tq = S + kNoAlloc.tq;
  bins.lb = reinterpret_cast<int*>(S + kNoAlloc.lb);
  bins.idx = reinterpret_cast<int*>(S + kNoAlloc.idx);
  bins.otq = S + kNoAlloc.otq;
  bins.ob = reinterpret_cast<int*>(S + kNoAlloc.ob);
  bins.oidx = reinterpret_cast<int*>(S + kNoAlloc.oidx);
  void* binpart = S + kNoAlloc.binpart;
  void* dwtab = S + kNoAlloc.wtab;

  cudaStream_t st = p->stream;
  const size_t es = p->fp64 ? 8 : 4;
  const size_t Mtot = (size_t)p->M[0] * p->M[1] * p->M[2];
  const size_t ss = esp::spread_smem_bytes(p->fp64, g), gs = esp::gather_smem_bytes(p->fp64, g);
  if (ss > 227 * 1024 || gs > 227 * 1024)
    return report(fail(p, ESP_ERR_ARG, "tile does not fit in shared memory"));
  ESP_CUDA(nullptr, esp::configure_kernels(p->fp64, w, ss, gs));
  int dev = 0, sms = 152, occ_s = 1, occ_g = 1;
  ESP_CUDA(nullptr, cudaGetDevice(&dev));
  ESP_CUDA(nullptr, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ESP_CUDA(nullptr, esp::occupancy(p->fp64, p->io_double, w, ss, gs, &occ_s, &occ_g));
  const int nblocks = std::max(1, std::min(p->ntiles, sms * std::max(occ_s, 1)));

  k_put_window_table<<<1, 256, 0, st>>>(targ, dwtab, p->fp64 ? 1 : 0);
  ESP_CUDA(nullptr, cudaGetLastError());
  // the array keeps the last call's contents: the counters and control words must start
  // at zero (a completed call leaves them zero, a failed one may not)
  ESP_CUDA(nullptr, cudaMemsetAsync(bins.count, 0, sizeof(int) * (size_t)p->ntiles, st));
  ESP_CUDA(nullptr, cudaMemsetAsync(bins.ctrl, 0, sizeof(int) * esp::kCtrl, st));
  ESP_CUDA(nullptr, cudaMemsetAsync(bins.hq, 0, sizeof(float) * esp::kHQ * (size_t)p->ntiles, st));
  ESP_CUDA(nullptr, esp::launch_bin(p->io_double, p->fp64, pos, q, n, g, bins, binpart,
                                    nullptr, 0, st));
  ESP_CUDA(nullptr, cudaMemsetAsync(grid_out, 0, es * Mtot, st));
  ESP_CUDA(nullptr, esp::launch_spread(p->fp64, g, p->ntiles, nblocks, bins, dwtab, grid_out, st));
  return ESP_OK;
}
