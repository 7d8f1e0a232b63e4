// Host driver and C ABI of the stage update (declared in include/fx.h).
//
// fx_grid_create builds, in FP64 on the host, the 1-d reconstruction/divergence tables of every
// direction from the coordinate moments <(x - x_c)^j> of each cell (Sec. 5.1, Eq. 14), the group
// edges and the Planck-series coefficients.  The caller provides all device memory (the
// workspace) at fx_bind_workspace; the library never allocates device memory itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/fx.h"
#include "fx_adjoint.cuh"
#include "fx_vterms.cuh"
#include "fx_layers.cuh"
#include "fx_launch.h"

using namespace fx;

namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// -------------------------------------------------------------------------------------------
// Coordinate moments of one cell, normalised: m_j = Int xi^j w dx / Int w dx, xi = x - x_c,
// for the 1-d volume weight w of a direction (Cartesian 1; spherical r: r^2 dr/dx1; theta:
// |sin theta|).  Closed-form series on the symmetric interval [-h/2, h/2].
// -------------------------------------------------------------------------------------------
// S_m = Int_{-h/2}^{h/2} xi^m dxi
double sym_power_integral(int m, double h) {
  if (m % 2) return 0.0;
  return 2.0 * std::pow(0.5 * h, m + 1) / (m + 1);
}

struct Moments { double w0, m1, m2; };

// weight exp(a xi) (times a constant): Int xi^j e^{a xi} = sum_k a^k/k! S_{j+k}
Moments moments_exp(double a, double h) {
  double M[3] = {0, 0, 0};
  for (int j = 0; j < 3; ++j) {
    double term = 1.0, s = 0.0;
    for (int k = 0; k < 60; ++k) {
      if (k > 0) term *= a / k;
      s += term * sym_power_integral(j + k, h);
    }
    M[j] = s;
  }
  return {M[0], M[1] / M[0], M[2] / M[0]};
}
// weight (x_c + xi)^2 (identity radial map)
Moments moments_r2(double xc, double h) {
  double M[3];
  for (int j = 0; j < 3; ++j)
    M[j] = xc * xc * sym_power_integral(j, h) + 2.0 * xc * sym_power_integral(j + 1, h) +
           sym_power_integral(j + 2, h);
  return {std::fabs(M[0]), M[1] / M[0], M[2] / M[0]};
}
// weight sin(theta_c + xi) = sin(theta_c) cos(xi) + cos(theta_c) sin(xi); the sign of the weight
// is constant on every cell (ghost cells beyond the axis mirror it), so normalised moments follow
Moments moments_sin(double tc, double h) {
  double M[3];
  for (int j = 0; j < 3; ++j) {
    double c = 0.0, s = 0.0, fc = 1.0, fs = 1.0;
    for (int k = 0; k < 30; ++k) {
      if (k > 0) { fc /= (2.0 * k - 1.0) * (2.0 * k); }
      fs = fc / (2.0 * k + 1.0);
      double sg = (k % 2) ? -1.0 : 1.0;
      c += sg * fc * sym_power_integral(j + 2 * k, h);
      s += sg * fs * sym_power_integral(j + 2 * k + 1, h);
    }
    M[j] = std::sin(tc) * c + std::cos(tc) * s;
  }
  return {std::fabs(M[0]), M[1] / M[0], M[2] / M[0]};
}

// 3x3 solve A^T y = e (returns the row vector e^T A^{-1}), Gaussian elimination with pivoting.
void solve_row(const double A[3][3], const double e[3], double y[3]) {
  double M[3][4];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) M[r][c] = A[c][r];
    M[r][3] = e[r];
  }
  for (int c = 0; c < 3; ++c) {
    int p = c;
    for (int r = c + 1; r < 3; ++r) if (std::fabs(M[r][c]) > std::fabs(M[p][c])) p = r;
    for (int q = 0; q < 4; ++q) std::swap(M[p][q], M[c][q]);
    for (int r = 0; r < 3; ++r) {
      if (r == c) continue;
      double f = M[r][c] / M[c][c];
      for (int q = c; q < 4; ++q) M[r][q] -= f * M[c][q];
    }
  }
  for (int r = 0; r < 3; ++r) y[r] = M[r][3] / M[r][r];
}

}  // namespace

struct PlanckTableHost;
struct fx_grid {
  fx_params P{};
  DevGrid dg{};
  int D = 0, G = 0, GP = 0, NV = 0;
  int64_t ncell = 0;
  std::vector<double> tab[3];  // [NTAB][n+4] per direction (FP64 master copy)
  GroupConst gc{};
  VtConst vtc{};
  LayerSet layers{};      // boundary layers (n = 0: none); the device copy sits at off_layers
  size_t off_layers = 0;
  double time = 0.0;      // time of the state (advanced by fx_step), for the layers' fronts
  PlanckParams pk{};
  // workspace layout (byte offsets)
  size_t ws_bytes = 0, off_status = 0, off_tab[3] = {0, 0, 0}, off_gc = 0, off_vtc = 0, off_A = 0, off_B = 0,
         off_tot = 0;
  size_t state_bytes = 0, elem = 8;
  unsigned char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int chunk = 32;
  fx_status sticky = FX_OK;
  std::string err;
  unsigned* h_status = nullptr;  // pinned
  std::vector<float4> ptab;       // FP32 Planck band tables [G][ptab_nu] (see PlanckTable)
  int ptab_nu = 0;
  float ptab_u0 = 0.0f;
  size_t off_ptab = 0;
  size_t off_hrow = 0;            // FP64 scale-factor rows T_HA, T_HB per direction (curvilinear)
  size_t off_faces = 0;           // gas face buffer [dir][NG+1 (+D-1 with vterms)][faces of dir]
  size_t off_opk = 0;             // opacity factors of the stage input [K, S][cells]
  size_t off_sflag = 0;           // shock flags of the stage input [cells] (carbuncle guard)
  int64_t face_off[3] = {0, 0, 0};
  int64_t faces_elems = 0;
  bool uniform[3] = {false, false, false};
  // per-kernel timing: one event triple (before the face kernel, between, after the stage
  // kernel) per stage launch since timing was enabled; events are pooled across reads
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t nev = 0;
  // objective (boundary radiation energy outflow, reading R19): per-row face fluxes of one stage
  // [rows][G] and FP64 accumulators obj[0] = J, obj[1] = dJ/dkappa0 (adjoint)
  bool objective = false;
  size_t off_phi = 0, off_obj = 0;
  size_t off_bud = 0;  // budgets (reading R13): rows of FP64 accumulators, see StageArgs::budget
  // One step (both stages) as a CUDA graph, replayed by fx_step while nothing that its launches
  // capture changes: the step, the workspace, the budgets flag, kappa0 and the march chunk (the
  // key).  Captured on the handle's own stream (capture is not available on the legacy default
  // stream), launched on the bound one.  Not used with boundary layers, per-kernel timing or the
  // objective (their launches change from step to step or need host events).
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t step_exec = nullptr;
  struct StepKey { double dt, kappa0; const void* ws; int budgets, chunk; } step_key{};
  bool graphs_ok = true;  // false after a capture failed: launch directly from then on
  bool budgets = false;  // accumulate the budgets during fx_step
  int64_t phi_rows = 0;
  double phi_area = 0.0;
  // adjoint: the forward pass records the stages of the last checkpoint segment in the adjoint
  // workspace, so that the backward pass need not recompute that segment.  The records are valid
  // for the workspace, step count, checkpoint interval and step recorded here (none: null).
  const void* adj_rec_ws = nullptr;
  int adj_rec_nsteps = 0, adj_rec_k = 0;
  double adj_rec_dt = 0.0;
};

namespace {

fx_status fail(fx_grid* h, fx_status s, const std::string& msg) {
  if (h) {
    if (h->sticky == FX_OK) h->sticky = s;
    h->err = msg;
  }
  return s;
}
fx_status cuda_fail(fx_grid* h, cudaError_t e, const char* where) {
  return fail(h, FX_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// The first out-of-range index that the index checks of the debug build recorded in the status
// region (words: bits, site, index, extent), as "index i outside [0, n) at file:line".
std::string bounds_message(const unsigned* w) {
  static const char* const files[] = {"fx_stage.cuh", "fx_gas.cuh",  "fx_couple.cuh", "fx_couple64.cuh",
                                      "fx_ye.cuh",    "fx_vterms.cuh", "fx_adjoint.cuh", "fx_layers.cuh",
                                      "fx_device.cuh", "fx_api.cu"};
  const unsigned tag = w[1] >> 16, line = w[1] & 0xffffu;
  std::string file = "tag " + std::to_string(tag);
  for (const char* f : files)
    if (fxb_file_tag(f) == tag) file = f;
  long long i, n;
  std::memcpy(&i, w + 2, sizeof i);
  std::memcpy(&n, w + 4, sizeof n);
  return "index " + std::to_string(i) + " outside [0, " + std::to_string(n) + ") at " + file + ":" +
         std::to_string(line) + " (index checks of the debug build)";
}

bool half_integer(double x) { return std::fabs(2.0 * x - std::round(2.0 * x)) < 1e-12; }

// Radial map r(x1) and its derivative (Appendix A).
double rmap(const fx_params& P, double x) {
  if (P.map1 == FX_MAP_EXP) return std::exp(x);
  if (P.map1 == FX_MAP_SINH) return P.map_rt * std::sinh(x / P.map_rt);
  return x;
}
double drmap(const fx_params& P, double x) {
  if (P.map1 == FX_MAP_EXP) return std::exp(x);
  if (P.map1 == FX_MAP_SINH) return std::cosh(x / P.map_rt);
  return 1.0;
}

// Moments of the radial volume weight r^2 dr/dx1 over a cell centred at xc of width h by
// Gauss-Legendre quadrature (16 points: two 8-point halves); the integrand is smooth and has no
// closed form that avoids cancellation near the origin for the sinh map.
Moments moments_quad(const fx_params& P, double xc, double h) {
  static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
  static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
  double M[3] = {0.0, 0.0, 0.0};
  for (int half = 0; half < 2; ++half) {
    const double c = xc + (half ? 0.25 : -0.25) * h, hw = 0.25 * h;
    for (int k = 0; k < 8; ++k) {
      const double xi = (k < 4 ? 1.0 : -1.0) * hw * xg[k % 4] + (c - xc);
      const double x = xc + xi, r = rmap(P, x), w = wg[k % 4] * hw * r * r * drmap(P, x);
      M[0] += w;
      M[1] += w * xi;
      M[2] += w * xi * xi;
    }
  }
  return {M[0], M[1] / M[0], M[2] / M[0]};
}

Moments cell_moments(const fx_params& P, int d, double xc, double h) {
  if (P.geom == FX_CART || d >= 2) return {h, 0.0, h * h / 12.0};
  if (d == 0) {
    if (P.map1 == FX_MAP_EXP) {
      Moments m = moments_exp(3.0, h);
      m.w0 *= std::exp(3.0 * xc);
      return m;
    }
    if (P.map1 == FX_MAP_SINH) return moments_quad(P, xc, h);
    return moments_r2(xc, h);
  }
  return moments_sin(xc, h);
}

// Build the reconstruction/divergence table of direction d (padded cells -2 .. n+1).
void build_table(const fx_params& P, int d, std::vector<double>& T) {
  const int n = (int)P.n[d], np = n + 4;
  const double h = (P.x_hi[d] - P.x_lo[d]) / n;
  T.assign((size_t)NTAB * np, 0.0);
  std::vector<Moments> mo(np + 2);
  std::vector<double> xc(np + 2);
  for (int i = -1; i <= np; ++i) {  // one extra cell on each side for the stencil of ghosts
    double c = P.x_lo[d] + (i - 2 + 0.5) * h;
    xc[i + 1] = c;
    mo[i + 1] = cell_moments(P, d, c, h);
  }
  auto put = [&](int e, int ip, double v) { T[(size_t)e * np + ip] = v; };
  for (int ip = 0; ip < np; ++ip) {
    // moments of cells ip-1, ip, ip+1 in the frame of cell ip (scaled by h)
    double mu1[3], mu2[3];
    for (int k = -1; k <= 1; ++k) {
      const Moments& m = mo[ip + 1 + k];
      double s = (xc[ip + 1 + k] - xc[ip + 1]) / h;
      double a1 = m.m1 / h, a2 = m.m2 / (h * h);
      mu1[k + 1] = s + a1;
      mu2[k + 1] = s * s + 2.0 * s * a1 + a2;
    }
    const double xl = -0.5, xr = 0.5;  // faces in units of h
    // system 1 (Eq. 15): face values as weights of the three averages
    double A1[3][3];
    for (int k = 0; k < 3; ++k) { A1[k][0] = 1.0; A1[k][1] = mu1[k]; A1[k][2] = mu2[k]; }
    double el[3] = {1.0, xl, xl * xl}, er[3] = {1.0, xr, xr * xr}, w[3];
    solve_row(A1, el, w);
    put(T_WA0, ip, w[0]); put(T_WA1, ip, w[1]); put(T_WA2, ip, w[2]);
    solve_row(A1, er, w);
    put(T_WB0, ip, w[0]); put(T_WB1, ip, w[1]); put(T_WB2, ip, w[2]);
    // face-interval reset (R2)
    double sL = (xl - mu1[0]) / (mu1[1] - mu1[0]);
    double sR = (xr - mu1[1]) / (mu1[2] - mu1[1]);
    put(T_SL2, ip, sL * sL); put(T_TL2, ip, (1.0 - sL) * (1.0 - sL));
    put(T_SR2, ip, sR * sR); put(T_TR2, ip, (1.0 - sR) * (1.0 - sR));
    // system 2 (Eq. 16): end slopes as weights of (a, mean, b)
    double A2[3][3] = {{1.0, xl, xl * xl}, {1.0, mu1[1], mu2[1]}, {1.0, xr, xr * xr}};
    double dl[3] = {0.0, 1.0, 2.0 * xl}, dr[3] = {0.0, 1.0, 2.0 * xr};
    solve_row(A2, dl, w);
    put(T_AL0, ip, w[0]); put(T_AL1, ip, w[1]); put(T_AL2, ip, w[2]);
    solve_row(A2, dr, w);
    put(T_AR0, ip, w[0]); put(T_AR1, ip, w[1]); put(T_AR2, ip, w[2]);
    double M2L = mu2[1] - 2.0 * xl * mu1[1] + xl * xl;
    double M2R = mu2[1] - 2.0 * xr * mu1[1] + xr * xr;
    put(T_RHL, ip, 1.0 / M2L);  // w^2 = 1 in units of h
    put(T_RHR, ip, 1.0 / M2R);
    // linear MC on centroid gaps (absolute units)
    put(T_IL, ip, 1.0 / (h * (mu1[1] - mu1[0])));
    put(T_IR, ip, 1.0 / (h * (mu1[2] - mu1[1])));
    put(T_IC, ip, 1.0 / (h * (mu1[2] - mu1[0])));
    put(T_DL, ip, h * (xl - mu1[1]));
    put(T_DR, ip, h * (xr - mu1[1]));
    // divergence factors, optical-depth length, scale factors, connection coefficients
    put(T_VOL, ip, mo[ip + 1].w0);
    const double xl_abs = xc[ip + 1] - 0.5 * h, xr_abs = xc[ip + 1] + 0.5 * h;
    const double ell = h * (mu1[1] - mu1[0]);  // centroid gap of the lower face
    for (int e : {T_XS, T_X1, T_X2, T_XH, T_HA, T_HB, T_QI, T_RI}) put(e, ip, 1.0);
    for (int e : {T_GA, T_GB, T_GC}) put(e, ip, 0.0);
    if (P.geom == FX_CART || d >= 2) {
      for (int e : {T_FL, T_FR, T_FL1, T_FR1, T_FL2, T_FR2}) put(e, ip, 1.0 / h);
      put(T_ELL, ip, ell);
      continue;
    }
    if (d == 0) {  // radius r(x1): faces carry r^2 (scalar), r^2 dr/dx1 (r comp.), r^3 (theta comp.)
      const double Vr = mo[ip + 1].w0;
      const double rl = rmap(P, xl_abs), rr = rmap(P, xr_abs);
      const double ql = drmap(P, xl_abs), qr = drmap(P, xr_abs);
      put(T_FL, ip, rl * rl / Vr);
      put(T_FR, ip, rr * rr / Vr);
      put(T_FL1, ip, rl * rl * ql / Vr);
      put(T_FR1, ip, rr * rr * qr / Vr);
      put(T_FL2, ip, rl * rl * rl / Vr);
      put(T_FR2, ip, rr * rr * rr / Vr);
      put(T_ELL, ip, ell * ql);
      // (interior faces have r > 0: the host rejects grids that reach r = 0; a ghost face of an
      // identity map may sit at r = 0, a row the velocity terms never read)
      put(T_QI, ip, 1.0 / ql);
      put(T_RI, ip, rl != 0.0 ? 1.0 / rl : 0.0);
      // theta faces of this radial cell: Int r dr/dx1, Int r (dr/dx1)^2, Int r^2 dr/dx1 over it
      auto gl = [&](auto f) {  // 8-point Gauss-Legendre on the cell
        static const double xg[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
        static const double wg[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
        double sum = 0.0, c = 0.5 * (xl_abs + xr_abs), hw = 0.5 * h;
        for (int k = 0; k < 4; ++k) sum += wg[k] * (f(c + hw * xg[k]) + f(c - hw * xg[k]));
        return sum * hw;
      };
      const double ra = gl([&](double x) { return std::fabs(rmap(P, x)) * drmap(P, x); });
      const double rb = gl([&](double x) { double q = drmap(P, x); return std::fabs(rmap(P, x)) * q * q; });
      const double rc = gl([&](double x) { double r = rmap(P, x); return r * r * drmap(P, x); });
      put(T_XS, ip, ra / Vr);
      put(T_X1, ip, rb / Vr);
      put(T_X2, ip, rc / Vr);
      put(T_XH, ip, rc / ra);
      // cell scale factors sqrt<g_11>, sqrt<g_22> (identity theta map: g_22 = r^2)
      put(T_HA, ip, std::sqrt(gl([&](double x) { double q = drmap(P, x), r = rmap(P, x); return q * q * std::fabs(r * r * q); }) / Vr));
      put(T_HB, ip, std::sqrt(gl([&](double x) { double q = drmap(P, x), r = rmap(P, x); return r * r * std::fabs(r * r * q); }) / Vr));
      const double g221 = gl([&](double x) { double q = drmap(P, x), r = rmap(P, x); return q / r * std::fabs(r * r * q); }) / Vr;
      const double g122 = -gl([&](double x) { double q = drmap(P, x), r = rmap(P, x); return r / q * std::fabs(r * r * q); }) / Vr;
      // pressure balance in r: <Gamma^1_11> = dA_1/dV - <Gamma^2_21> - <Gamma^3_31>
      const double g111 = (rr * rr * qr - rl * rl * ql) / Vr - 2.0 * g221;
      put(T_GA, ip, g111);
      put(T_GB, ip, g221);
      put(T_GC, ip, g122);
    } else {  // polar angle theta = x2 (identity map), weight |sin theta|
      const double Th = mo[ip + 1].w0;
      const double sl = std::fabs(std::sin(xl_abs)), sr = std::fabs(std::sin(xr_abs));
      for (int e : {T_FL, T_FL1, T_FL2}) put(e, ip, sl / Th);
      for (int e : {T_FR, T_FR1, T_FR2}) put(e, ip, sr / Th);
      put(T_ELL, ip, ell);
      // Eq. 79f: <cot theta>, Int cos over the cell with the weight's sign (mirror cells flip it)
      const double sgn = std::sin(xc[ip + 1]) >= 0.0 ? 1.0 : -1.0;
      const double g332 = sgn * (std::sin(xr_abs) - std::sin(xl_abs)) / Th;
      put(T_GA, ip, (sr - sl) / Th - g332);  // Eq. 85: <Gamma^2_22> = dA_2/dV - <Gamma^3_32>
      put(T_GB, ip, g332);
    }
  }
}

// Bernoulli numbers over factorials b_k = B_k/k! from the generating function t/(e^t - 1):
// sum_{j=0}^{k} b_j / (k+1-j)! = 0 for k >= 1.
void planck_coefficients(PlanckParams& pk) {
  const int K = 2 * NPLANCK_LO + 2;
  std::vector<double> b(K + 1, 0.0), ifact(K + 3, 1.0);
  for (int i = 1; i <= K + 2; ++i) ifact[i] = ifact[i - 1] / i;
  b[0] = 1.0;
  for (int k = 1; k <= K; ++k) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += b[j] * ifact[k + 1 - j];
    b[k] = -s;  // the j = k term has coefficient 1/1!
  }
  for (int m = 1; m <= NPLANCK_LO; ++m) {
    pk.c64.lo[m - 1] = b[2 * m] / (2.0 * m + 3.0);
    pk.c64.wd[m - 1] = b[2 * m];
  }
  for (int n = 1; n <= NPLANCK_UP; ++n) pk.c64.rn[n - 1] = 1.0 / n;
  for (int m = 1; m <= NPLANCK_LO32; ++m) {
    pk.lo32[m - 1] = (float)pk.c64.lo[m - 1];
    pk.wd32[m - 1] = (float)pk.c64.wd[m - 1];
  }
}

// Host FP64 Planck integrals for the FP32 band tables: D(x) = Int_0^x (Bernoulli series in
// b_k = B_k/k!, x < XSPLIT) and P(x) = Int_x^inf (exponential series), as on the device.
double host_planck_lower(const PlanckParams& pk, double x) {
  double x2 = x * x, sd = 0.0;
  for (int m = NPLANCK_LO - 1; m >= 0; --m) sd = sd * x2 + pk.c64.lo[m];
  return x2 * x * (1.0 / 3.0 - 0.125 * x + x2 * sd);
}
double host_planck_upper(double x) {
  double y = std::exp(-x), yn = y, s = 0.0;
  for (int n = 1; n <= 200; ++n) {
    double rn = 1.0 / n;
    double t = yn * rn * (x * x * x + rn * (3.0 * x * x + rn * (6.0 * x + 6.0 * rn)));
    s += t;
    if (t <= 1e-18 * s) break;
    yn *= y;
  }
  return s;
}
double host_band(const PlanckParams& pk, double a, double b) {
  const double total = std::pow(M_PI, 4) / 15.0;
  bool alo = a < XSPLIT, blo = b < XSPLIT;
  if (alo && blo) return host_planck_lower(pk, b) - host_planck_lower(pk, a);
  if (!alo && !blo) return host_planck_upper(a) - host_planck_upper(b);
  return (total - host_planck_lower(pk, a)) - host_planck_upper(b);
}
double host_w(double x) { return x > 700.0 ? 0.0 : x * x * x * x / std::expm1(x); }

}  // namespace
struct PlanckTableHost { std::vector<float4> tab; int nu = 0; float u0 = 0.0f; };
namespace {

void build_planck_table(const fx_params& P, const GroupConst& gc, const PlanckParams& pk,
                        PlanckTableHost& T) {
  const int G = P.ngroups;
  const double u0 = std::floor(std::log2(P.eps_min / PTAB_XMAX));
  const double u1 = std::ceil(std::log2(P.eps_max / PTAB_XMIN));
  T.nu = (int)((u1 - u0) * PTAB_PER_OCT) + 2;
  T.u0 = (float)u0;
  T.tab.assign((size_t)G * T.nu, make_float4(0.0f, 0.0f, 0.0f, 0.0f));
  const double h = 1.0 / PTAB_PER_OCT;
  for (int g = 0; g < G; ++g)
    for (int i = 0; i < T.nu; ++i) {
      const double Tt = std::exp2(u0 + i * h);
      const double a = gc.edge[g] / Tt, b = gc.edge[g + 1] / Tt;
      const double I = host_band(pk, a, b);
      double L, m;
      if (I > std::exp2(-200.0)) {
        L = std::log2(I);
        m = h * (host_w(a) - host_w(b)) / I;  // h dL/du, L = log2 I, u = log2 T
      } else {
        L = -200.0;
        m = -h * a;  // the band underflows in FP32 here; keep the table smooth and negative
      }
      const double k = std::floor(L);
      // 2^floor(L), exact in FP32 down to the smallest normal number (0 below, where the band
      // integral flushes to zero in FP32 anyway)
      const float sc = k >= -126.0 ? (float)std::ldexp(1.0, (int)k) : 0.0f;
      T.tab[(size_t)g * T.nu + i] = make_float4((float)(L - k), (float)m, (float)k, sc);
    }
}

// Layout of the device Planck table, a measured choice (interaction kernel per launch, node-major
// against group-major): kh2d (2-d, 16 groups) 0.142 against 0.156 ms; lognormal3d (3-d, 12
// groups) 3.77 against 3.47 ms; blobs2d (2-d, 8 groups) 0.033 against 0.029 ms.  A warp's cells
// read nodes i and i+1 of every group: group-major keeps the lanes' nodes of one group on one
// cache line when their temperatures differ, node-major keeps a lane's groups together.
bool ptab_node_major(const fx_grid* h) { return h->D <= 2 && h->P.ngroups >= 16; }

// The FP64 scale-factor rows T_HA, T_HB of every direction, as k_init_equilibrium reads them.
std::vector<double> hrows(const fx_grid* h) {
  std::vector<double> out;
  for (int d = 0; d < h->D; ++d) {
    const size_t np = (size_t)h->P.n[d] + 4;
    for (int e : {T_HA, T_HB}) out.insert(out.end(), h->tab[d].begin() + e * np, h->tab[d].begin() + (e + 1) * np);
  }
  return out;
}

template <class R> const R* dev_tab(const fx_grid* h, int d) {
  return reinterpret_cast<const R*>(h->ws + h->off_tab[d]);
}

// ------------------------------------------------------------------ helper kernels
// Cells c0 .. c0 + nc - 1 from primitive rows of stride ps (row r of cell c at prim[r ps + c - c0]).
// hrow (null on Cartesian grids): per direction d, the FP64 rows T_HA and T_HB of its table
// (n_d + 4 entries each, padded), whose products over the directions are the cell's scale factors
// h_0, h_1: the momentum is covariant, rho vhat_q h_q.
template <class R>
__global__ void k_init_equilibrium(const double* prim, int64_t c0, int64_t nc, int64_t ps, R* out, DevGrid g,
                                   const GroupConst* gcp, PlanckParams pk, const double* hrow) {
  const int64_t ncell = g.ncell;
  const int G = g.G, D = g.D, NG = 2 + D;
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nc * (G + 1)) return;
  const int64_t cl = t / (G + 1), c = c0 + cl;
  int j = (int)(t % (G + 1));
  double rho = prim[cl], p = prim[ps + cl], Tr = prim[(int64_t)(2 + D) * ps + cl];
  if (j == G) {  // gas of this cell (and, with three species, rho Y_e from prim row 3 + D)
    double ke = 0.0;
    out[c] = (R)rho;
    if (g.species > 1) out[(int64_t)(NG + (1 + D) * G) * ncell + c] = (R)(rho * prim[(int64_t)(3 + D) * ps + cl]);
    double hq[3] = {1.0, 1.0, 1.0};
    if (hrow) {
      const int64_t i3[3] = {c % g.n[0], (c / g.n[0]) % g.n[1], c / ((int64_t)g.n[0] * g.n[1])};
      const double* r = hrow;
      for (int d = 0; d < D; ++d) {
        const int np = g.n[d] + 4;
        hq[0] *= r[i3[d] + 2];
        hq[1] *= r[np + i3[d] + 2];
        r += 2 * np;
      }
    }
    for (int q = 0; q < D; ++q) {
      double vh = prim[(int64_t)(2 + q) * ps + cl];
      out[(int64_t)(1 + q) * ncell + c] = (R)(rho * vh * (q < 2 ? hq[q] : 1.0));
      ke += 0.5 * rho * vh * vh;
    }
    out[(int64_t)(NG - 1) * ncell + c] = (R)(p / (g.gamma - 1.0) + ke);
    return;
  }
  const GroupConst& gc = *gcp;
  double invT = 1.0 / Tr;
  const int gg = j % g.Gs, sp = j / g.Gs;  // group and species of channel j
  PlanckEdge<double> lo = planck_edge64(gc.edge[gg] * invT, pk.c64);
  PlanckEdge<double> hi = planck_edge64(gc.edge[gg + 1] * invT, pk.c64);
  double B = g.a_rad * 0.15398973382026502 * Tr * Tr * Tr * Tr * planck_band(lo, hi);
  if (g.species > 1) {  // equilibrium weight 2 Y_e, 2 (1 - Y_e), 1
    const double Ye = prim[(int64_t)(3 + D) * ps + cl];
    B *= sp == 0 ? 2.0 * Ye : (sp == 1 ? 2.0 * (1.0 - Ye) : 1.0);
  }
  out[(int64_t)NG * ncell + c * G + j] = (R)B;
  for (int q = 0; q < D; ++q) out[(int64_t)NG * ncell + ((int64_t)(1 + q) * ncell + c) * G + j] = R(0);
}

template <class S, class T>
__global__ void k_convert(const S* in, T* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (T)in[i];
}

// Neumaier pair
struct KS { double s, c; };
__device__ __forceinline__ void ks_add(KS& a, double x) {
  double t = a.s + x;
  if (fabs(a.s) >= fabs(x)) a.c += (a.s - t) + x; else a.c += (x - t) + a.s;
  a.s = t;
}
__device__ __forceinline__ void ks_merge(KS& a, const KS& b) {
  ks_add(a, b.s);
  a.c += b.c;
}

constexpr int TOT_BLOCKS = 512, TOT_THREADS = 256;

template <class R>
__global__ void __launch_bounds__(TOT_THREADS)
k_totals_partial(const R* U, DevGrid g, const double* vol0, const double* vol1, const double* vol2,
                 double* part) {
  const int64_t ncell = g.ncell;
  const int G = g.G, D = g.D, NG = 2 + D;
  const double ic2 = 1.0 / (g.c * g.c);
  KS acc[FX_NTOTALS];
  for (int q = 0; q < FX_NTOTALS; ++q) acc[q] = {0.0, 0.0};
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int ix = (int)(c % g.n[0]);
    int iy = (int)((c / g.n[0]) % g.n[1]);
    int iz = (int)(c / ((int64_t)g.n[0] * g.n[1]));
    double V = vol0[ix + 2] * (D > 1 ? vol1[iy + 2] : 1.0) * (D > 2 ? vol2[iz + 2] : 1.0);
    double Es = 0.0, Fs[3] = {0.0, 0.0, 0.0};
    const R* E = U + (int64_t)NG * ncell + c * G;
    for (int j = 0; j < G; ++j) Es += (double)E[j];
    for (int q = 0; q < D; ++q) {
      const R* F = U + (int64_t)NG * ncell + ((int64_t)(1 + q) * ncell + c) * G;
      for (int j = 0; j < G; ++j) Fs[q] += (double)F[j];
    }
    ks_add(acc[0], V * (double)U[c]);
    for (int q = 0; q < D; ++q) ks_add(acc[1 + q], V * ((double)U[(int64_t)(1 + q) * ncell + c] + Fs[q] * ic2));
    ks_add(acc[4], V * ((double)U[(int64_t)(NG - 1) * ncell + c] + Es));
    ks_add(acc[5], V * Es);
  }
  __shared__ KS sh[TOT_THREADS];
  for (int q = 0; q < FX_NTOTALS; ++q) {
    sh[threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = TOT_THREADS / 2; s > 0; s >>= 1) {
      if ((int)threadIdx.x < s) ks_merge(sh[threadIdx.x], sh[threadIdx.x + s]);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      part[(blockIdx.x * FX_NTOTALS + q) * 2 + 0] = sh[0].s;
      part[(blockIdx.x * FX_NTOTALS + q) * 2 + 1] = sh[0].c;
    }
    __syncthreads();
  }
}

__global__ void k_totals_final(const double* part, int nblocks, double* out) {
  int q = threadIdx.x;
  if (q >= FX_NTOTALS) return;
  KS a = {0.0, 0.0};
  for (int b = 0; b < nblocks; ++b) {
    KS p = {part[(b * FX_NTOTALS + q) * 2 + 0], part[(b * FX_NTOTALS + q) * 2 + 1]};
    ks_merge(a, p);
  }
  out[q] = a.s + a.c;
}

// acc[0] += w * sum(x[0..n)) in FP64, deterministic: one block of 1024 threads, strided partial
// sums, then a fixed shuffle and shared-memory tree.
template <class T>
__global__ void __launch_bounds__(1024) k_sum_into(const T* x, int64_t n, double w, double* acc) {
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += (double)x[i];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  __shared__ double sh[32];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double b = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x == 0) acc[0] += w * b;
  }
}

// dJ/drho(x, 0) at fixed pressure, velocity and radiation (reading R20): with U = (rho, rho v,
// p/(gamma-1) + rho |v|^2/2, E, F), dU/drho = (1, v, |v|^2/2, 0, 0).
template <class R>
__global__ void k_grad_rho(const R* U, const R* lam, DevGrid g, R* out) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int64_t n = g.ncell;
  const R rho = U[c];
  R s = lam[c], v2 = R(0);
  for (int q = 0; q < g.D; ++q) {
    const R v = U[(1 + q) * n + c] / rho;
    s += lam[(1 + q) * n + c] * v;
    v2 += v * v;
  }
  out[c] = s + lam[(1 + g.D) * n + c] * R(0.5) * v2;
}

template <class R>
__global__ void k_set_density(R* U, const R* rho_new, DevGrid g) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const int64_t n = g.ncell;
  const R rho = U[c], rn = rho_new[c];
  R v2 = R(0);
  for (int q = 0; q < g.D; ++q) {
    const R v = U[(1 + q) * n + c] / rho;
    U[(1 + q) * n + c] = rn * v;
    v2 += v * v;
  }
  U[(1 + g.D) * n + c] += R(0.5) * (rn - rho) * v2;
  U[c] = rn;
}

bool has_ws(fx_grid* h) { return h && h->ws; }

// Per-launch scalar constants, computed once in FP64 and rounded to the kernel types.
template <class T>
Consts<T> make_consts(const fx_grid* h, double dt, double dts, double alpha, bool fp32_newton) {
  const fx_params& P = h->P;
  Consts<T> k;
  k.gamma = (T)P.gamma;
  k.gm1 = (T)(P.gamma - 1.0);
  k.cv = (T)(1.0 / (P.gamma - 1.0));
  k.c = (T)P.c_light;
  k.ic2 = (T)(1.0 / (P.c_light * P.c_light));
  k.hc = (T)(0.5 * P.c_light);
  k.hc2 = (T)(0.5 * P.c_light * P.c_light);
  k.kappa0 = (T)P.kappa0;
  k.sigma0 = (T)P.sigma0;
  k.rho_floor = (T)P.rho_floor;
  k.u_floor = (T)(P.p_floor / (P.gamma - 1.0));
  k.E_floor = (T)std::max(P.E_floor, sizeof(T) == 4 ? 1e-37 : 1e-300);
  k.aN = (T)(P.a_rad * 15.0 / std::pow(M_PI, 4));
  k.cdts = (T)(P.c_light * dts);
  k.dt = (T)dt;
  k.alpha = (T)alpha;
  k.beta = (T)(1.0 - alpha);
  // FP32 iterates stop at FP32 resolution (the paper's own tolerance is 1e-6, Sec. 5.3)
  k.rtol = (T)(fp32_newton ? std::max(P.newton_rtol, 2e-7) : P.newton_rtol);
  k.atol = (T)(fp32_newton ? 1e-7 : 1e-14);
  for (int d = 0; d < 3; ++d) k.idx[d] = (T)h->dg.inv_dx[d];
  return k;
}

// Stage arguments common to every stage of a handle (tables, constants, buffers).
template <class R>
StageArgs<R> stage_args(fx_grid* h) {
  StageArgs<R> a{};
  a.g = h->dg;
  for (int d = 0; d < 3; ++d) a.tab[d] = dev_tab<R>(h, d < h->D ? d : 0);
  a.gc = reinterpret_cast<const GroupConst*>(h->ws + h->off_gc);
  a.vtc = reinterpret_cast<const VtConst*>(h->ws + h->off_vtc);
  a.faces = reinterpret_cast<const R*>(h->ws + h->off_faces);
  a.faces_out = reinterpret_cast<R*>(h->ws + h->off_faces);
  a.opk = reinterpret_cast<R*>(h->ws + h->off_opk);
  a.sflag = h->P.shock_guard > 0.0 ? reinterpret_cast<unsigned char*>(h->ws + h->off_sflag) : nullptr;
  for (int d = 0; d < 3; ++d) {
    a.face_off[d] = h->face_off[d];
    a.uniform[d] = d < h->D && h->uniform[d];
    for (int e = 0; e < NTAB; ++e)
      a.urow[d][e] = d < h->D ? (R)h->tab[d][(size_t)e * (h->P.n[d] + 4)] : R(0);
  }
  a.ptab.tab = reinterpret_cast<const float4*>(h->ws + h->off_ptab);
  a.ptab.nu = h->ptab_nu;
  a.ptab.u0 = h->ptab_u0;
  a.ptab.si = ptab_node_major(h) ? h->P.ngroups : 1;
  a.ptab.sg = ptab_node_major(h) ? 1 : h->ptab_nu;
  a.pk = h->pk;
  a.status = reinterpret_cast<unsigned*>(h->ws + h->off_status);
#ifdef FX_BOUNDS_CHECK
  a.ptab.n = (int)h->ptab.size();
  a.ptab.status = a.status;
  a.n_state = h->ncell * h->NV;
  a.n_faces = h->faces_elems;
#endif
  a.chunk = h->chunk;
  a.phi_area = (R)h->phi_area;
  return a;
}

// Set the stage-dependent fields: stage 1 (U1 = U0 + dt L(U0), interaction with dt) or stage 2
// (U = U0/2 + (U1 + dt L(U1))/2, interaction with dt/2; reading R10).
template <class R>
void set_stage(fx_grid* h, StageArgs<R>& a, int stage, double dt) {
  const bool f32n = sizeof(R) == 4;  // FP32 group sums bound the attainable residual
  a.dt = dt;
  a.bw_flux = 0.5 * dt;                // both stages' fluxes enter U^(n+1) with weight dt/2
  a.bw_cpl = stage == 1 ? 0.5 : 1.0;   // U^(1) enters U^(n+1) with weight 1/2
  if (stage == 1) {
    a.dts = dt;
    a.alpha = 0.0;
    a.kd = make_consts<double>(h, dt, dt, 0.0, f32n);
    a.kf = make_consts<float>(h, dt, dt, 0.0, f32n);
  } else {
    a.dts = 0.5 * dt;
    a.alpha = 0.5;
    a.kd = make_consts<double>(h, dt, 0.5 * dt, 0.5, f32n);
    a.kf = make_consts<float>(h, dt, 0.5 * dt, 0.5, f32n);
  }
}

// Enqueue one stage (both kernels), with the per-kernel timing events when enabled and the
// objective's reduction when a.phi_out is set.
template <class R, class NT>
fx_status launch_one_stage(fx_grid* h, const StageArgs<R>& a, const char* what) {
  cudaEvent_t e4[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  if (h->timing) {
    while (h->ev.size() < h->nev + 4) {
      cudaEvent_t x;
      e = cudaEventCreate(&x);
      if (e != cudaSuccess) return cuda_fail(h, e, "timing event");
      h->ev.push_back(x);
    }
    for (int q = 0; q < 4; ++q) e4[q] = h->ev[h->nev + q];
    h->nev += 4;
    e = cudaEventRecord(e4[0], h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing event");
  }
  switch (h->D) {
    case 1: e = launch_stage<R, 1, NT, false>(a, h->GP, h->stream, e4[1], e4[2]); break;
    case 2:
      e = h->P.geom == FX_SPH ? launch_stage<R, 2, NT, true>(a, h->GP, h->stream, e4[1], e4[2])
                              : launch_stage<R, 2, NT, false>(a, h->GP, h->stream, e4[1], e4[2]);
      break;
    default: e = launch_stage<R, 3, NT, false>(a, h->GP, h->stream, e4[1], e4[2]); break;
  }
  if (e == cudaSuccess && e4[3]) e = cudaEventRecord(e4[3], h->stream);
  if (e == cudaSuccess && a.phi_out) {
    // J += dt/2 Phi(U_in): this stage's share of the RK-weighted boundary outflow
    k_sum_into<R><<<1, 1024, 0, h->stream>>>(a.phi_out, h->phi_rows * h->G, 0.5 * a.dt,
                                             reinterpret_cast<double*>(h->ws + h->off_obj));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(h, e, what);
  return FX_OK;
}

// Boundary layers of state U at the step's time + toff, and the end-of-step advance of the
// layers' time (no status set: the caller reports a failed launch).
template <class R>
cudaError_t launch_layers(fx_grid* h, R* U, double toff, cudaStream_t st) {
  if (h->layers.n == 0) return cudaSuccess;
  int nmax = 1;
  for (int q = 0; q < h->layers.n; ++q) {
    const LayerDev& L = h->layers.L[q];
    const int64_t nb = (int64_t)(L.hi[0] - L.lo[0]) * (L.hi[1] - L.lo[1]) * (L.hi[2] - L.lo[2]);
    nmax = std::max(nmax, (int)std::min<int64_t>((nb + LAYER_THREADS - 1) / LAYER_THREADS, 4096));
  }
  const LayerSet* ls = reinterpret_cast<const LayerSet*>(h->ws + h->off_layers);
  layer_kernel<R><<<dim3((unsigned)nmax, (unsigned)h->layers.n, 1), LAYER_THREADS, 0, st>>>(ls, U, h->dg, toff);
  return cudaGetLastError();
}
inline cudaError_t launch_layer_advance(fx_grid* h, double dt, cudaStream_t st) {
  if (h->layers.n == 0) return cudaSuccess;
  layer_advance<<<1, 32, 0, st>>>(reinterpret_cast<LayerSet*>(h->ws + h->off_layers), dt);
  return cudaGetLastError();
}

// One step's launches (stage 1, stage 2) captured as a CUDA graph on the handle's own stream;
// null when the stream, the capture or the instantiation fails (fx_step then launches directly;
// the failure sets no sticky status).
template <class R, class NT>
cudaGraphExec_t capture_step(fx_grid* h, const StageArgs<R>& a1, const StageArgs<R>& a2) {
  if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->cap_stream = nullptr;
    (void)cudaGetLastError();
    return nullptr;
  }
  auto launch = [&](const StageArgs<R>& a) -> cudaError_t {
    switch (h->D) {
      case 1: return launch_stage<R, 1, NT, false>(a, h->GP, h->cap_stream, nullptr, nullptr);
      case 2:
        return h->P.geom == FX_SPH ? launch_stage<R, 2, NT, true>(a, h->GP, h->cap_stream, nullptr, nullptr)
                                   : launch_stage<R, 2, NT, false>(a, h->GP, h->cap_stream, nullptr, nullptr);
      default: return launch_stage<R, 3, NT, false>(a, h->GP, h->cap_stream, nullptr, nullptr);
    }
  };
  // the step waits for the bound stream's earlier work through the graph launch itself
  if (cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  R* A = const_cast<R*>(a1.in);
  R* B = a1.out;
  const double dt = a1.dt;
  cudaError_t e = launch_layers<R>(h, A, 0.0, h->cap_stream);
  if (e == cudaSuccess) e = launch(a1);
  if (e == cudaSuccess) e = launch_layers<R>(h, B, dt, h->cap_stream);
  if (e == cudaSuccess) e = launch(a2);
  if (e == cudaSuccess) e = launch_layers<R>(h, A, dt, h->cap_stream);
  if (e == cudaSuccess) e = launch_layer_advance(h, dt, h->cap_stream);
  cudaGraph_t gph = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(h->cap_stream, &gph);
  if (e == cudaSuccess) e = ee;
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess && gph) e = cudaGraphInstantiate(&ex, gph, 0);
  if (gph) cudaGraphDestroy(gph);
  if (e != cudaSuccess || !ex) {
    if (ex) cudaGraphExecDestroy(ex);
    (void)cudaGetLastError();
    return nullptr;
  }
  return ex;
}

template <class R, class NT>
fx_status enqueue_steps(fx_grid* h, double dt, int nsteps) {
  StageArgs<R> a = stage_args<R>(h);
  R* A = reinterpret_cast<R*>(h->ws + h->off_A);
  R* B = reinterpret_cast<R*>(h->ws + h->off_B);
  if (h->objective) a.phi_out = reinterpret_cast<R*>(h->ws + h->off_phi);
  if (h->budgets) {
    a.budget = reinterpret_cast<double*>(h->ws + h->off_bud);
    for (int d = 0; d < h->D; ++d)
      if (h->P.bc_lo[d] != FX_PERIODIC || h->P.bc_hi[d] != FX_PERIODIC) a.budget_bnd = 1;
  }
  StageArgs<R> a1 = a, a2 = a;
  set_stage(h, a1, 1, dt);
  set_stage(h, a2, 2, dt);
  a1.in = A; a1.base = nullptr; a1.out = B;
  a2.in = B; a2.base = A; a2.out = A;
  // boundary layers: the stage-1 input at the step's time t, the stage-2 input and the result at
  // t + dt; then t advances on the device
  auto layers = [&](R* U, double toff) -> fx_status {
    const cudaError_t e = launch_layers<R>(h, U, toff, h->stream);
    return e == cudaSuccess ? FX_OK : cuda_fail(h, e, "boundary layer launch");
  };
  if (h->graphs_ok && !h->timing && !a.phi_out && nsteps > 0) {
    const fx_grid::StepKey key{dt, h->P.kappa0, h->ws, h->budgets ? 1 : 0, h->chunk};
    if (h->step_exec && std::memcmp(&key, &h->step_key, sizeof(key)) != 0) {
      cudaGraphExecDestroy(h->step_exec);
      h->step_exec = nullptr;
    }
    if (!h->step_exec) {
      h->step_exec = capture_step<R, NT>(h, a1, a2);
      h->step_key = key;
      if (!h->step_exec) h->graphs_ok = false;
    }
    if (h->step_exec) {
      for (int s = 0; s < nsteps; ++s) {
        const cudaError_t e = cudaGraphLaunch(h->step_exec, h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "step graph launch");
        h->time += dt;
      }
      return FX_OK;
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    fx_status st = layers(A, 0.0);
    if (st != FX_OK) return st;
    st = launch_one_stage<R, NT>(h, a1, "stage 1 launch");
    if (st != FX_OK) return st;
    if ((st = layers(B, dt)) != FX_OK) return st;
    st = launch_one_stage<R, NT>(h, a2, "stage 2 launch");
    if (st != FX_OK) return st;
    if ((st = layers(A, dt)) != FX_OK) return st;
    const cudaError_t e = launch_layer_advance(h, dt, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "boundary layer launch");
    h->time += dt;
  }
  return FX_OK;
}

// ---- adjoint (config of the boundary-outflow objective; Cartesian grids)

// Adjoint workspace layout for nsteps steps with a checkpoint every k steps.
struct AdjLayout {
  size_t S = 0, Tn = 0, LWn = 0;
  int nseg = 0, k = 0;
  size_t off_ckpt = 0, off_U = 0, off_U1 = 0, off_pre1 = 0, off_pre2 = 0, off_t1 = 0, off_t2 = 0,
         off_LA = 0, off_LB = 0, off_LP = 0, off_LW = 0, off_kpart = 0, bytes = 0;
  unsigned nblk = 0;
};
AdjLayout adj_layout(const fx_grid* h, int nsteps, int k) {
  AdjLayout L;
  L.k = k;
  L.nseg = nsteps > 0 ? (nsteps + k - 1) / k : 1;
  L.S = align_up(h->state_bytes);
  L.Tn = align_up((size_t)h->ncell * h->elem);
  L.LWn = align_up((size_t)h->ncell * (2 + h->D + h->G * (1 + h->D) + h->G) * h->elem);
  L.nblk = adj_cell_blocks(h->ncell, h->GP);
  size_t off = 0;
  L.off_ckpt = off; off += (size_t)L.nseg * L.S;
  L.off_U = off; off += (size_t)(k + 1) * L.S;   // U[0] unused (the checkpoint), U[1..k]
  L.off_U1 = off; off += (size_t)k * L.S;
  L.off_pre1 = off; off += (size_t)k * L.S;
  L.off_pre2 = off; off += (size_t)k * L.S;
  L.off_t1 = off; off += (size_t)k * L.Tn;
  L.off_t2 = off; off += (size_t)k * L.Tn;
  L.off_LA = off; off += L.S;
  L.off_LB = off; off += L.S;
  L.off_LP = off; off += L.S;
  L.off_LW = off; off += L.LWn;
  L.off_kpart = off; off += align_up((size_t)L.nblk * sizeof(double));
  L.bytes = off;
  return L;
}

// Pass 1 (forward): from the current state, nsteps steps with the objective, a checkpoint of
// the state every k steps (checkpoint 0 = the current state); the handle's state is unchanged.
// The steps of the last segment also record each stage's pre-interaction state and temperature.
// Pass 2 (backward): segment by segment from the last checkpoint, recompute the segment's
// steps recording each stage's pre-interaction state and temperature (except for the last
// segment when the forward pass of the same workspace recorded it), then run the stage adjoints
// backwards through it.  seed scales the objective (the adjoint of J).
template <class R, class NT>
fx_status adjoint_impl(fx_grid* h, double dt, int nsteps, int k, unsigned char* ws, bool fwd, bool bwd,
                       double seed, void* grad_state, void* grad_rho, double* J, double* dJ_dkappa0) {
  const AdjLayout L = adj_layout(h, nsteps, k);
  cudaStream_t st = h->stream;
  auto P = [&](size_t off) { return reinterpret_cast<R*>(ws + off); };
  auto ckpt = [&](int j) { return P(L.off_ckpt + (size_t)j * L.S); };
  auto Ub = [&](int m) { return P(L.off_U + (size_t)m * L.S); };
  auto U1b = [&](int m) { return P(L.off_U1 + (size_t)m * L.S); };
  auto pre1 = [&](int m) { return P(L.off_pre1 + (size_t)m * L.S); };
  auto pre2 = [&](int m) { return P(L.off_pre2 + (size_t)m * L.S); };
  auto t1 = [&](int m) { return P(L.off_t1 + (size_t)m * L.Tn); };
  auto t2 = [&](int m) { return P(L.off_t2 + (size_t)m * L.Tn); };
  R* LA = P(L.off_LA);
  R* LB = P(L.off_LB);
  R* LP = P(L.off_LP);
  R* LW = P(L.off_LW);
  double* kpart = reinterpret_cast<double*>(ws + L.off_kpart);
  double* obj = reinterpret_cast<double*>(h->ws + h->off_obj);
  cudaError_t e;
  StageArgs<R> a = stage_args<R>(h);
  StageArgs<R> a1 = a, a2 = a;
  set_stage(h, a1, 1, dt);
  set_stage(h, a2, 2, dt);
  const bool tim = h->timing;
  h->timing = false;
  if (fwd) {
    h->adj_rec_ws = nullptr;
    e = cudaMemsetAsync(obj, 0, sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ckpt(0), h->ws + h->off_A, h->state_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) { h->timing = tim; return cuda_fail(h, e, "adjoint setup"); }
    a1.phi_out = a2.phi_out = reinterpret_cast<R*>(h->ws + h->off_phi);
    R* cur = ckpt(0);
    const int last0 = (L.nseg - 1) * k;  // first step of the last segment
    for (int n = 0; n < nsteps; ++n) {
      if (n >= last0) {
        // last segment: the layout and records of the backward pass's recomputation
        const int m = n - last0;
        R* Um = m == 0 ? ckpt(L.nseg - 1) : Ub(m);
        a1.in = Um; a1.base = nullptr; a1.out = U1b(m); a1.pre_out = pre1(m); a1.tstar_out = t1(m);
        a2.in = U1b(m); a2.base = Um; a2.out = Ub(m + 1); a2.pre_out = pre2(m); a2.tstar_out = t2(m);
      } else {
        R* nxt = ((n + 1) % k == 0 && n + 1 < nsteps) ? ckpt((n + 1) / k) : Ub(n & 1);
        a1.in = cur; a1.base = nullptr; a1.out = U1b(0);
        a2.in = U1b(0); a2.base = cur; a2.out = nxt;
        cur = nxt;
      }
      fx_status s1 = launch_one_stage<R, NT>(h, a1, "adjoint forward pass");
      if (s1 == FX_OK) s1 = launch_one_stage<R, NT>(h, a2, "adjoint forward pass");
      if (s1 != FX_OK) { h->timing = tim; return s1; }
    }
    a1.phi_out = a2.phi_out = nullptr;
    a1.pre_out = a2.pre_out = nullptr;
    a1.tstar_out = a2.tstar_out = nullptr;
    if (nsteps > 0) {
      h->adj_rec_ws = ws;
      h->adj_rec_nsteps = nsteps;
      h->adj_rec_k = k;
      h->adj_rec_dt = dt;
    }
    if (J) {
      e = cudaMemcpyAsync(J, obj, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { h->timing = tim; return cuda_fail(h, e, "objective read"); }
    }
  }
  if (!bwd) { h->timing = tim; return FX_OK; }

  // reverse sweep, one checkpoint segment at a time
  AdjArgs<R> b{};
  b.g = h->dg;
  for (int d = 0; d < 3; ++d) {
    b.tab[d] = a.tab[d];
    b.uniform[d] = a.uniform[d];
    for (int q = 0; q < NTAB; ++q) b.urow[d][q] = a.urow[d][q];
  }
  b.gc = a.gc;
  b.pk = a.pk;
  b.ptab = a.ptab;
#ifdef FX_BOUNDS_CHECK
  b.status = a.status;
  b.n_state = a.n_state;
#endif
  b.lam_w = LW;
  b.kpart = kpart;
  b.phi_area = (R)h->phi_area;
  b.dt = dt;
  b.wJ = (R)(0.5 * dt * seed);
  AdjArgs<R> b1 = b, b2 = b;
  b1.alpha = 0.0; b1.kd = a1.kd; b1.kf = a1.kf;
  b2.alpha = 0.5; b2.kd = a2.kd; b2.kf = a2.kf;
  e = cudaMemsetAsync(LA, 0, h->state_bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(obj + 1, 0, sizeof(double), st);
  if (e != cudaSuccess) { h->timing = tim; return cuda_fail(h, e, "adjoint setup"); }
  auto run = [&](AdjArgs<R>& bb) -> cudaError_t {
    cudaError_t x;
    switch (h->D) {
      case 1: x = adj_launch_couple<R, 1>(bb, h->GP, st); break;
      case 2: x = adj_launch_couple<R, 2>(bb, h->GP, st); break;
      default: x = adj_launch_couple<R, 3>(bb, h->GP, st); break;
    }
    if (x != cudaSuccess) return x;
    k_sum_into<double><<<1, 1024, 0, st>>>(kpart, L.nblk, 1.0, obj + 1);
    x = cudaMemsetAsync(LW, 0, L.LWn, st);
    if (x != cudaSuccess) return x;
    switch (h->D) {
      case 1: x = adj_launch_face<R, 1>(bb, st); break;
      case 2: x = adj_launch_face<R, 2>(bb, st); break;
      default: x = adj_launch_face<R, 3>(bb, st); break;
    }
    if (x != cudaSuccess) return x;
    switch (h->D) {
      case 1: x = adj_launch_cell<R, 1>(bb, h->GP, st); break;
      case 2: x = adj_launch_cell<R, 2>(bb, h->GP, st); break;
      default: x = adj_launch_cell<R, 3>(bb, h->GP, st); break;
    }
    if (x != cudaSuccess) return x;
    k_sum_into<double><<<1, 1024, 0, st>>>(kpart, L.nblk, 1.0, obj + 1);
    return cudaGetLastError();
  };
  const bool recorded = h->adj_rec_ws == ws && h->adj_rec_nsteps == nsteps && h->adj_rec_k == k &&
                        h->adj_rec_dt == dt;
  for (int j = L.nseg - 1; j >= 0 && nsteps > 0; --j) {
    const int s0 = j * k, s1 = std::min(s0 + k, nsteps), ns = s1 - s0;
    // recompute the segment, recording each stage's pre-interaction state and temperature (the
    // forward pass recorded the last one); recomputing overwrites the last segment's records
    const bool have = recorded && j == L.nseg - 1;
    if (!have) h->adj_rec_ws = nullptr;
    for (int m = 0; m < ns && !have; ++m) {
      R* Um = m == 0 ? ckpt(j) : Ub(m);
      a1.in = Um; a1.base = nullptr; a1.out = U1b(m); a1.pre_out = pre1(m); a1.tstar_out = t1(m);
      a2.in = U1b(m); a2.base = Um; a2.out = Ub(m + 1); a2.pre_out = pre2(m); a2.tstar_out = t2(m);
      fx_status s2 = launch_one_stage<R, NT>(h, a1, "adjoint recomputation");
      if (s2 == FX_OK) s2 = launch_one_stage<R, NT>(h, a2, "adjoint recomputation");
      if (s2 != FX_OK) { h->timing = tim; return s2; }
    }
    for (int m = ns - 1; m >= 0; --m) {
      R* Um = m == 0 ? ckpt(j) : Ub(m);
      // stage 2: lam(U^(n+1)) = LA -> lam(U^(1)) = LB, lam(U^n) partial = LA
      b2.in = U1b(m); b2.pre = pre2(m); b2.tstar = t2(m); b2.lam_out = LA; b2.lam_pre = LP;
      b2.lam_in = LB; b2.lam_base = LA; b2.accumulate_in = 0;
      e = run(b2);
      if (e != cudaSuccess) { h->timing = tim; return cuda_fail(h, e, "adjoint stage 2"); }
      // stage 1: lam(U^(1)) = LB -> lam(U^n) += ...
      b1.in = Um; b1.pre = pre1(m); b1.tstar = t1(m); b1.lam_out = LB; b1.lam_pre = LP;
      b1.lam_in = LA; b1.lam_base = nullptr; b1.accumulate_in = 1;
      e = run(b1);
      if (e != cudaSuccess) { h->timing = tim; return cuda_fail(h, e, "adjoint stage 1"); }
    }
  }
  h->timing = tim;
  if (grad_state) {
    e = cudaMemcpyAsync(grad_state, LA, h->state_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "gradient copy");
  }
  if (grad_rho) {
    k_grad_rho<R><<<(unsigned)((h->ncell + 255) / 256), 256, 0, st>>>(ckpt(0), LA, h->dg, (R*)grad_rho);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "density gradient");
  }
  double res = 0.0;
  e = cudaMemcpyAsync(&res, obj + 1, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint result");
  if (dJ_dkappa0) *dJ_dkappa0 = res;
  return FX_OK;
}

}  // namespace

extern "C" {

fx_status fx_grid_create(const fx_params* params, fx_grid** out, size_t* workspace_bytes) {
  if (out) *out = nullptr;
  if (!params || !out || !workspace_bytes) return FX_ERR_ARG;
  const fx_params& P = *params;
  if (P.dims < 1 || P.dims > 3) return FX_ERR_ARG;
  if (P.ngroups < 1 || P.ngroups > MAXG) return FX_ERR_UNSUPPORTED;
  for (int d = 0; d < P.dims; ++d) {
    if (P.n[d] < 4 || P.n[d] > (int64_t)1 << 30) return FX_ERR_ARG;
    if (!(P.x_hi[d] > P.x_lo[d])) return FX_ERR_ARG;
    for (int s = 0; s < 2; ++s) {
      int bc = s ? P.bc_hi[d] : P.bc_lo[d];
      if (bc < FX_OUTFLOW || bc > FX_AXIS) return FX_ERR_ARG;
    }
    if ((P.bc_lo[d] == FX_PERIODIC) != (P.bc_hi[d] == FX_PERIODIC)) return FX_ERR_ARG;
  }
  if (P.geom != FX_CART && P.geom != FX_SPH) return FX_ERR_ARG;
  if (P.geom == FX_SPH) {
    // spherical (r, theta) grids: 2-d, radial map identity or exponential, theta in [0, pi]
    if (P.dims != 2 || (P.map1 != FX_MAP_ID && P.map1 != FX_MAP_EXP && P.map1 != FX_MAP_SINH))
      return FX_ERR_UNSUPPORTED;
    if (P.map1 == FX_MAP_SINH && !(P.map_rt > 0.0)) return FX_ERR_ARG;
    if (P.x_lo[1] < 0.0 || P.x_hi[1] > M_PI + 1e-12) return FX_ERR_ARG;
    if (P.map1 != FX_MAP_EXP && !(P.x_lo[0] > 0.0)) return FX_ERR_UNSUPPORTED;
  }
  if (P.precision != FX_FP64 && P.precision != FX_FP32 && P.precision != FX_FP32_F64NEWTON)
    return FX_ERR_ARG;
  if (P.rad_recon_order != 1 && P.rad_recon_order != 2) return FX_ERR_ARG;
  if (P.riemann < FX_HLLC || P.riemann > FX_LLF || !(P.shock_guard >= 0.0)) return FX_ERR_ARG;
  if (P.vterms != 0 && P.vterms != 1) return FX_ERR_ARG;
  if (P.species != 0 && P.species != 1 && P.species != 3) return FX_ERR_ARG;
  const int NS = P.species > 1 ? P.species : 1;  // species
  if (NS > 1) {
    if (!(P.xi0 >= 0.0) || !std::isfinite(P.xi0)) return FX_ERR_ARG;
    // three species: 3 ngroups <= 32 channels
    if (NS * P.ngroups > MAXG) return FX_ERR_UNSUPPORTED;
  }
  const int NCH = NS * P.ngroups;  // radiation channels
  if (!(P.gamma > 1.0) || !(P.c_light > 0.0) || !(P.a_rad > 0.0)) return FX_ERR_ARG;
  if (!half_integer(P.kap_rho_exp) || !half_integer(P.kap_T_exp)) return FX_ERR_UNSUPPORTED;
  if (!(P.eps_min > 0.0) || !(P.eps_max > P.eps_min)) return FX_ERR_ARG;
  if (P.newton_maxit < 1 || P.bisect_maxit < 0 || !(P.newton_rtol > 0.0)) return FX_ERR_ARG;
  if (!(P.rho_floor > 0.0) || !(P.p_floor > 0.0) || !(P.E_floor > 0.0)) return FX_ERR_ARG;
  {
    const int GP = NCH <= 8 ? 8 : (NCH <= 16 ? 16 : 32);
    size_t smem = 0;
    if (P.precision == FX_FP64)
      smem = P.dims == 1 ? stage_smem<double, 1>(GP, NCH)
           : P.dims == 2 ? stage_smem<double, 2>(GP, NCH) : stage_smem<double, 3>(GP, NCH);
    else
      smem = P.dims == 1 ? stage_smem<float, 1>(GP, NCH)
           : P.dims == 2 ? stage_smem<float, 2>(GP, NCH) : stage_smem<float, 3>(GP, NCH);
    if (smem > 227 * 1024) return FX_ERR_UNSUPPORTED;  // per-block shared memory of sm_103a
  }

  fx_grid* h = new fx_grid();
  h->P = P;
  h->D = P.dims;
  h->G = NCH;
  h->GP = NCH <= 8 ? 8 : (NCH <= 16 ? 16 : 32);
  h->NV = 2 + P.dims + NCH * (1 + P.dims) + (NS > 1 ? 1 : 0);  // + the composition block
  h->ncell = 1;
  for (int d = 0; d < P.dims; ++d) h->ncell *= P.n[d];
  h->elem = P.precision == FX_FP64 ? 8 : 4;
  // kernels index the state and the gas face buffer with 32-bit element offsets
  if ((double)h->ncell * h->NV >= 4294967295.0 || (double)h->ncell * (3 + P.dims) * P.dims * 1.01 >= 4294967295.0) {
    delete h;
    return FX_ERR_UNSUPPORTED;
  }

  DevGrid& g = h->dg;
  g.D = P.dims;
  g.G = NCH;
  g.species = NS;
  g.Gs = P.ngroups;
  g.xi0 = P.xi0;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < P.dims ? (int)P.n[d] : 1;
    g.bc_lo[d] = d < P.dims ? P.bc_lo[d] : FX_PERIODIC;
    g.bc_hi[d] = d < P.dims ? P.bc_hi[d] : FX_PERIODIC;
  }
  g.geom = P.geom;
  g.rad_order = P.rad_recon_order;
  g.ncell = h->ncell;
  g.gamma = P.gamma;
  g.c = P.c_light;
  g.a_rad = P.a_rad;
  g.kappa0 = P.kappa0;
  g.sigma0 = P.sigma0;
  g.kap_rho_h = (int)std::lround(2.0 * P.kap_rho_exp);
  g.kap_T_h = (int)std::lround(2.0 * P.kap_T_exp);
  g.rho_floor = P.rho_floor;
  g.p_floor = P.p_floor;
  g.E_floor = P.E_floor;
  g.newton_maxit = P.newton_maxit;
  g.bisect_maxit = P.bisect_maxit;
  g.newton_rtol = P.newton_rtol;
  g.couple = P.couple;
  g.riemann = P.riemann;
  g.shock_guard = P.shock_guard;
  g.vterms = P.vterms;
  for (int d = 0; d < 3; ++d)
    g.inv_dx[d] = d < P.dims ? (double)P.n[d] / (P.x_hi[d] - P.x_lo[d]) : 1.0;

  for (int d = 0; d < P.dims; ++d) build_table(P, d, h->tab[d]);
  // group edges; the opacity factor eps_g^d per channel (channel k is group k % ngroups)
  for (int j = 0; j <= P.ngroups; ++j)
    h->gc.edge[j] = P.eps_min * std::pow(P.eps_max / P.eps_min, (double)j / P.ngroups);
  for (int j = 0; j < h->G; ++j) {
    const int gg = j % P.ngroups;
    h->gc.efac[j] = std::pow(std::sqrt(h->gc.edge[gg] * h->gc.edge[gg + 1]), P.kap_eps_exp);
  }
  for (int j = 0; j <= MAXG; ++j) h->gc.edge32[j] = (float)h->gc.edge[j];
  vt_constants(h->gc.edge, P.ngroups, h->vtc);
  for (int j = 0; j < MAXG; ++j) h->gc.efac32[j] = (float)h->gc.efac[j];
  planck_coefficients(h->pk);
  {
    PlanckTableHost T;
    build_planck_table(P, h->gc, h->pk, T);
    h->ptab.swap(T.tab);
    h->ptab_nu = T.nu;
    h->ptab_u0 = T.u0;
  }

  // chunk length along the march axis: 32 planes until the workspace is bound, where it is fitted
  // to the device (choose_chunk)
  if (P.dims >= 2) h->chunk = std::min((int)P.n[P.dims - 1], 32);
  // workspace layout
  size_t off = 0;
  h->off_status = off; off = align_up(off + 64);
  for (int d = 0; d < P.dims; ++d) { h->off_tab[d] = off; off = align_up(off + h->tab[d].size() * h->elem); }
  h->off_gc = off; off = align_up(off + sizeof(GroupConst));
  {
    size_t nh = 0;
    for (int d = 0; d < P.dims; ++d) nh += 2 * (size_t)(P.n[d] + 4);
    h->off_hrow = off; off = align_up(off + nh * sizeof(double));
  }
  h->off_vtc = off; off = align_up(off + sizeof(VtConst));
  h->off_ptab = off; off = align_up(off + h->ptab.size() * sizeof(float4));
  {
    int64_t fo = 0;
    for (int d = 0; d < P.dims; ++d) {
      h->face_off[d] = fo;
      // fluxes and v*, then (velocity terms on) the D - 1 transverse face velocities
      fo += (int64_t)(2 + P.dims + 1 + (P.vterms ? P.dims - 1 : 0)) * faces_along(g.n, d);
    }
    h->off_faces = off;
    h->faces_elems = fo;
    off = align_up(off + (size_t)fo * h->elem);
  }
  h->off_opk = off;
  off = align_up(off + (size_t)2 * h->ncell * h->elem);
  h->off_sflag = off;  // carbuncle guard: shock flags, one byte per cell
  off = align_up(off + (P.shock_guard > 0.0 ? (size_t)h->ncell : 0));
  // directions whose table rows are all equal (uniform Cartesian spacing) read one row
  for (int d = 0; d < P.dims; ++d) {
    const int np = (int)P.n[d] + 4;
    bool uni = true;
    for (int e = 0; e < NTAB && uni; ++e)
      for (int i = 1; i < np && uni; ++i) uni = h->tab[d][(size_t)e * np + i] == h->tab[d][(size_t)e * np];
    h->uniform[d] = uni;
  }
  h->state_bytes = (size_t)h->ncell * h->NV * h->elem;
  h->off_A = off; off = align_up(off + h->state_bytes);
  h->off_B = off; off = align_up(off + h->state_bytes);
  h->off_tot = off; off = align_up(off + (size_t)(TOT_BLOCKS * FX_NTOTALS * 2 + FX_NTOTALS) * sizeof(double));
  size_t vol_bytes = 0;
  for (int d = 0; d < P.dims; ++d) vol_bytes += align_up((size_t)(P.n[d] + 4) * sizeof(double));
  off += vol_bytes;
  // objective: one row of upper-x boundary faces per (y, z) line; Cartesian face area
  h->phi_rows = (P.dims > 1 ? P.n[1] : 1) * (P.dims > 2 ? P.n[2] : 1);
  h->phi_area = 1.0;
  for (int d = 1; d < P.dims; ++d) h->phi_area *= (P.x_hi[d] - P.x_lo[d]) / (double)P.n[d];
  h->off_phi = off; off = align_up(off + (size_t)h->phi_rows * h->G * h->elem);
  h->off_obj = off; off = align_up(off + 8 * sizeof(double));
  h->off_bud = off; off = align_up(off + (size_t)BUDGET_SLOTS * NBUDGET * sizeof(double));
  h->off_layers = off; off = align_up(off + sizeof(LayerSet));
  h->ws_bytes = off;
  *workspace_bytes = off;
  *out = h;
  return FX_OK;
}

size_t fx_state_elems(const fx_grid* h) { return h ? (size_t)h->ncell * h->NV : 0; }

int fx_march_chunk(const fx_grid* h) { return h ? (h->D >= 2 ? h->chunk : 0) : -1; }

fx_status fx_budgets_enable(fx_grid* h, int on) {
  if (!h) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  h->budgets = on != 0;
  cudaError_t e = cudaMemsetAsync(h->ws + h->off_bud, 0, (size_t)BUDGET_SLOTS * NBUDGET * sizeof(double), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "budget reset");
  return FX_OK;
}

fx_status fx_budgets(fx_grid* h, double out[FX_NBUDGET]) {
  if (!h || !out) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  std::vector<double> rows((size_t)BUDGET_SLOTS * NBUDGET);
  cudaError_t e = cudaMemcpyAsync(rows.data(), h->ws + h->off_bud, rows.size() * sizeof(double),
                                  cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "budget read");
  for (int q = 0; q < NBUDGET; ++q) {
    double sum = 0.0;
    for (int r = 0; r < BUDGET_SLOTS; ++r) sum += rows[(size_t)r * NBUDGET + q];
    out[q] = sum;
  }
  return FX_OK;
}

fx_status fx_boundary_layers(fx_grid* h, const fx_layer* layers, int n, double t0) {
  if (!h || n < 0 || n > MAX_LAYERS || (n > 0 && !layers) || !std::isfinite(t0)) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  if (n > 0 && h->P.geom != FX_CART) return fail(h, FX_ERR_UNSUPPORTED, "boundary layers need a Cartesian grid");
  if (n > 0 && h->dg.species > 1) return fail(h, FX_ERR_UNSUPPORTED, "boundary layers carry no composition");
  const int D = h->D, G = h->G, NG = 2 + D;
  const int64_t nn[3] = {h->P.n[0], D > 1 ? h->P.n[1] : 1, D > 2 ? h->P.n[2] : 1};
  LayerSet S{};
  S.n = n;
  for (int d = 0; d < 3; ++d) {
    S.x_lo[d] = d < D ? h->P.x_lo[d] : 0.0;
    S.dx[d] = d < D ? (h->P.x_hi[d] - h->P.x_lo[d]) / (double)h->P.n[d] : 1.0;
  }
  for (int q = 0; q < n; ++q) {
    const fx_layer& L = layers[q];
    if (L.kind != FX_LAYER_FRONT && L.kind != FX_LAYER_MIRROR) return fail(h, FX_ERR_ARG, "layer kind");
    for (int d = 0; d < 3; ++d)
      if (L.lo[d] < 0 || L.hi[d] > nn[d] || L.lo[d] >= L.hi[d]) return fail(h, FX_ERR_ARG, "layer box outside the grid or empty");
    for (int r = 0; r < q; ++r) {  // boxes must not overlap
      const fx_layer& O = layers[r];
      bool sep = false;
      for (int d = 0; d < 3; ++d) sep = sep || L.hi[d] <= O.lo[d] || O.hi[d] <= L.lo[d];
      if (!sep) return fail(h, FX_ERR_ARG, "layer boxes overlap");
    }
    LayerDev& Ld = S.L[q];
    Ld.kind = L.kind;
    for (int d = 0; d < 3; ++d) { Ld.lo[d] = (int)L.lo[d]; Ld.hi[d] = (int)L.hi[d]; }
    if (L.kind == FX_LAYER_MIRROR) {
      if (L.d < 0 || L.d >= D) return fail(h, FX_ERR_ARG, "mirror direction");
      Ld.d = L.d;
      Ld.m = L.m;
    } else {
      Ld.x0 = L.x0; Ld.y0 = L.y0; Ld.cot = L.cot_alpha; Ld.speed = L.speed;
      // conserved states from the primitives (rho, p, v_1..v_D, T_rad): E_g = B_g(T_rad), F = 0
      const double* P2[2] = {L.A, L.B};
      double* U2[2] = {Ld.UA, Ld.UB};
      for (int w = 0; w < 2; ++w) {
        const double* pr = P2[w];
        if (!(pr[0] > 0.0) || !(pr[1] > 0.0) || !(pr[2 + D] > 0.0)) return fail(h, FX_ERR_ARG, "layer state");
        double ke = 0.0;
        U2[w][0] = pr[0];
        for (int d = 0; d < D; ++d) {
          U2[w][1 + d] = pr[0] * pr[2 + d];
          ke += 0.5 * pr[0] * pr[2 + d] * pr[2 + d];
        }
        U2[w][NG - 1] = pr[1] / (h->P.gamma - 1.0) + ke;
        const double T = pr[2 + D];
        for (int k = 0; k < G; ++k)
          U2[w][NG + k] = h->P.a_rad * 0.15398973382026502 * T * T * T * T *
                          host_band(h->pk, h->gc.edge[k] / T, h->gc.edge[k + 1] / T);
      }
    }
  }
  // every mirror source lies in the grid and outside every box
  for (int q = 0; q < n; ++q) {
    const fx_layer& L = layers[q];
    if (L.kind != FX_LAYER_MIRROR) continue;
    for (int64_t i = L.lo[L.d]; i < L.hi[L.d]; ++i) {
      const int64_t si = 2 * (int64_t)L.m - 1 - i;
      if (si < 0 || si >= nn[L.d]) return fail(h, FX_ERR_ARG, "mirror source outside the grid");
      for (int r = 0; r < n; ++r) {
        const fx_layer& O = layers[r];
        // the mirror images of the box's cells along d form the box with [si] in place of [i]
        int64_t lo[3] = {L.lo[0], L.lo[1], L.lo[2]}, hi[3] = {L.hi[0], L.hi[1], L.hi[2]};
        lo[L.d] = si; hi[L.d] = si + 1;
        bool sep = false;
        for (int d = 0; d < 3; ++d) sep = sep || hi[d] <= O.lo[d] || O.hi[d] <= lo[d];
        if (!sep) return fail(h, FX_ERR_ARG, "a mirror reads a layer box");
      }
    }
  }
  S.t = t0;
#ifdef FX_BOUNDS_CHECK
  S.status = reinterpret_cast<unsigned*>(h->ws + h->off_status);
  S.n_state = h->ncell * h->NV;
#endif
  h->layers = S;
  h->time = t0;
  if (h->step_exec) {  // a captured step holds the previous layer launches
    cudaGraphExecDestroy(h->step_exec);
    h->step_exec = nullptr;
  }
  cudaError_t e = cudaMemcpyAsync(h->ws + h->off_layers, &h->layers, sizeof(LayerSet), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "boundary layer upload");
  return FX_OK;
}

int fx_launches_per_step(const fx_grid* h) {
  if (!h) return 0;
  const bool split = h->P.couple != 0;  // the interaction kernel runs in every form
  return 2 * (2 + (split ? 1 : 0) + (h->objective ? 1 : 0) + (h->P.shock_guard > 0.0 ? 1 : 0) +
              (h->P.vterms ? 1 : 0) + (h->dg.species > 1 ? 1 : 0)) + (h->layers.n > 0 ? 4 : 0);
}

fx_status fx_objective_enable(fx_grid* h, int on) {
  if (!h) return FX_ERR_ARG;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  if (on && h->P.geom != FX_CART) return fail(h, FX_ERR_UNSUPPORTED, "the outflow objective needs a Cartesian grid");
  h->objective = on != 0;
  cudaError_t e = cudaMemsetAsync(h->ws + h->off_obj, 0, sizeof(double), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "objective reset");
  return FX_OK;
}

fx_status fx_boundary_energy_out(fx_grid* h, double* J) {
  if (!h || !J) return FX_ERR_ARG;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  cudaError_t e = cudaMemcpyAsync(J, h->ws + h->off_obj, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "objective read");
  return FX_OK;
}

fx_status fx_set_kappa0(fx_grid* h, double kappa0) {
  if (!h || !(kappa0 >= 0.0)) return FX_ERR_ARG;
  h->P.kappa0 = kappa0;
  h->dg.kappa0 = kappa0;
  return FX_OK;
}

fx_status fx_adjoint_workspace_bytes(const fx_grid* h, int nsteps, int k, size_t* bytes) {
  if (!h || !bytes || nsteps < 0 || k < 1) return FX_ERR_ARG;
  *bytes = adj_layout(h, nsteps, k).bytes;
  return FX_OK;
}

static fx_status adjoint_entry(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                               bool fwd, bool bwd, double seed, void* grad_state, void* grad_rho,
                               double* J, double* dJ_dkappa0) {
  if (!h) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  if (!(dt > 0.0) || nsteps < 0 || k < 1) return fail(h, FX_ERR_ARG, "dt must be > 0, nsteps >= 0, k >= 1");
  if (h->P.geom != FX_CART) return fail(h, FX_ERR_UNSUPPORTED, "the adjoint supports Cartesian grids");
  if (h->P.rad_recon_order != 1)
    return fail(h, FX_ERR_UNSUPPORTED, "the adjoint supports the linear radiation reconstruction");
  if (h->P.riemann != FX_HLLC || h->P.shock_guard > 0.0)
    return fail(h, FX_ERR_UNSUPPORTED, "the adjoint supports HLLC without the carbuncle guard");
  if (h->P.vterms)
    return fail(h, FX_ERR_UNSUPPORTED, "the adjoint does not include the velocity-dependent terms");
  if (h->layers.n > 0) return fail(h, FX_ERR_UNSUPPORTED, "the adjoint does not include boundary layers");
  if (h->dg.species > 1) return fail(h, FX_ERR_UNSUPPORTED, "the adjoint supports one radiation species");
  if (!adj_ws || adj_bytes < adj_layout(h, nsteps, k).bytes || (reinterpret_cast<uintptr_t>(adj_ws) % kAlign) != 0)
    return fail(h, FX_ERR_WORKSPACE, "adjoint workspace missing, too small or not 256-byte aligned");
  unsigned char* ws = static_cast<unsigned char*>(adj_ws);
  fx_status st;
  if (h->elem == 8)
    st = adjoint_impl<double, double>(h, dt, nsteps, k, ws, fwd, bwd, seed, grad_state, grad_rho, J, dJ_dkappa0);
  else if (h->P.precision == FX_FP32_F64NEWTON)
    st = adjoint_impl<float, double>(h, dt, nsteps, k, ws, fwd, bwd, seed, grad_state, grad_rho, J, dJ_dkappa0);
  else
    st = adjoint_impl<float, float>(h, dt, nsteps, k, ws, fwd, bwd, seed, grad_state, grad_rho, J, dJ_dkappa0);
  if (st != FX_OK) return st;
  return fx_sync(h);
}

fx_status fx_adjoint_forward(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                             double* J) {
  return adjoint_entry(h, dt, nsteps, k, adj_ws, adj_bytes, true, false, 1.0, nullptr, nullptr, J, nullptr);
}

fx_status fx_adjoint_backward(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                              double seed, void* grad_state, void* grad_rho, double* dJ_dkappa0) {
  return adjoint_entry(h, dt, nsteps, k, adj_ws, adj_bytes, false, true, seed, grad_state, grad_rho,
                       nullptr, dJ_dkappa0);
}

fx_status fx_adjoint(fx_grid* h, double dt, int nsteps, int k, void* adj_ws, size_t adj_bytes,
                     void* grad_state, void* grad_rho, double* J, double* dJ_dkappa0) {
  return adjoint_entry(h, dt, nsteps, k, adj_ws, adj_bytes, true, true, 1.0, grad_state, grad_rho, J,
                       dJ_dkappa0);
}

// Replace the density of the current state, holding pressure, velocity and radiation fixed
// (reading R20): m = rho_new v, rho e = rho e - rho |v|^2/2 + rho_new |v|^2/2.
fx_status fx_state_set_density(fx_grid* h, const void* rho, int rho_precision, int rho_is_device) {
  if (!h || !rho) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  const int my = h->elem == 8 ? FX_FP64 : FX_FP32;
  if (rho_precision != my) return fail(h, FX_ERR_ARG, "density precision must match the state");
  const size_t nb = (size_t)h->ncell * h->elem;
  // stage the new density in the second state buffer (free between steps)
  cudaError_t e = cudaMemcpyAsync(h->ws + h->off_B, rho, nb, rho_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "density upload");
  const unsigned blocks = (unsigned)((h->ncell + 255) / 256);
  if (h->elem == 8)
    k_set_density<double><<<blocks, 256, 0, h->stream>>>((double*)(h->ws + h->off_A), (const double*)(h->ws + h->off_B), h->dg);
  else
    k_set_density<float><<<blocks, 256, 0, h->stream>>>((float*)(h->ws + h->off_A), (const float*)(h->ws + h->off_B), h->dg);
  e = cudaGetLastError();
  if (e == cudaSuccess && !rho_is_device) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "density update");
  return FX_OK;
}

// March chunk of the stage kernel (planes per block), fitted to the bound device: it minimises
// (waves of blocks) x (planes per block + the prologue's share), with the device's multiprocessor
// count and the kernel's resident blocks per multiprocessor.  A grid that overshoots a whole
// number of waves by a little runs its last wave mostly empty; longer chunks spread the
// prologue (three planes loaded, two march reconstructions) over more planes.
fx_status choose_chunk(fx_grid* h) {
  if (h->D < 2) return FX_OK;
  int dev = 0, nsm = 0, nb = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    const int p = h->P.precision;
    const bool sph = h->P.geom == FX_SPH;
    if (h->D == 2 && sph)
      e = p == FX_FP64 ? stage_blocks_per_sm<double, 2, double, true>(h->GP, h->G, h->P.rad_recon_order, &nb)
        : p == FX_FP32 ? stage_blocks_per_sm<float, 2, float, true>(h->GP, h->G, h->P.rad_recon_order, &nb)
                       : stage_blocks_per_sm<float, 2, double, true>(h->GP, h->G, h->P.rad_recon_order, &nb);
    else if (h->D == 2)
      e = p == FX_FP64 ? stage_blocks_per_sm<double, 2, double, false>(h->GP, h->G, h->P.rad_recon_order, &nb)
        : p == FX_FP32 ? stage_blocks_per_sm<float, 2, float, false>(h->GP, h->G, h->P.rad_recon_order, &nb)
                       : stage_blocks_per_sm<float, 2, double, false>(h->GP, h->G, h->P.rad_recon_order, &nb);
    else
      e = p == FX_FP64 ? stage_blocks_per_sm<double, 3, double, false>(h->GP, h->G, h->P.rad_recon_order, &nb)
        : p == FX_FP32 ? stage_blocks_per_sm<float, 3, float, false>(h->GP, h->G, h->P.rad_recon_order, &nb)
                       : stage_blocks_per_sm<float, 3, double, false>(h->GP, h->G, h->P.rad_recon_order, &nb);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query");
  const int nm = (int)h->P.n[h->D - 1];
  const int ngl = groups_per_lane(h->elem == 4, h->D, h->GP);
  const int TC = tile_cells(h->D, h->GP / ngl, ngl);  // cells per tile
  const int TX = h->D == 3 ? (TC >= 16 ? TC / 4 : TC / 2) : TC, TY = TC / TX;
  int64_t tiles = (h->P.n[0] + TX - 1) / TX;
  if (h->D == 3) tiles *= (h->P.n[1] + TY - 1) / TY;
  const double slots = (double)std::max(nsm, 1) * std::max(nb, 1);
  double best = 1e300;
  int bc = std::min(nm, 32);
  for (int c = 8; c <= std::min(nm, 128); ++c) {
    const double waves = std::ceil((double)(tiles * ((nm + c - 1) / c)) / slots);
    const double cost = waves * (c + 1.5);
    if (cost < best) { best = cost; bc = c; }
  }
  h->chunk = bc;
  return FX_OK;
}

fx_status fx_bind_workspace(fx_grid* h, void* dev_ptr, size_t bytes, void* cuda_stream) {
  if (!h) return FX_ERR_ARG;
  if (!dev_ptr || bytes < h->ws_bytes || (reinterpret_cast<uintptr_t>(dev_ptr) % kAlign) != 0)
    return fail(h, FX_ERR_WORKSPACE, "workspace missing, too small or not 256-byte aligned");
  h->ws = static_cast<unsigned char*>(dev_ptr);
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  if (h->step_exec) {  // its launches point into the previous workspace
    cudaGraphExecDestroy(h->step_exec);
    h->step_exec = nullptr;
  }
  cudaError_t e;
  if (!h->h_status) {
    e = cudaMallocHost(&h->h_status, 6 * sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(h, e, "pinned status word");
  }
  e = cudaMemsetAsync(h->ws + h->off_status, 0, 64, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "status reset");
  e = cudaMemsetAsync(h->ws + h->off_bud, 0, (size_t)BUDGET_SLOTS * NBUDGET * sizeof(double), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->ws + h->off_obj, 0, 8 * sizeof(double), h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "budget reset");
  {
    const fx_status cs = choose_chunk(h);
    if (cs != FX_OK) return cs;
  }
  for (int d = 0; d < h->D; ++d) {
    const std::vector<double>& T = h->tab[d];
    if (h->elem == 8) {
      e = cudaMemcpyAsync(h->ws + h->off_tab[d], T.data(), T.size() * 8, cudaMemcpyHostToDevice, h->stream);
    } else {
      std::vector<float> f(T.begin(), T.end());
      e = cudaMemcpyAsync(h->ws + h->off_tab[d], f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "table upload");
  }
  // FP64 cell volumes for the totals (after the totals scratch)
  size_t off = h->off_tot + align_up((size_t)(TOT_BLOCKS * FX_NTOTALS * 2 + FX_NTOTALS) * sizeof(double));
  std::vector<double> vol;
  for (int d = 0; d < h->D; ++d) {
    const int np = (int)h->P.n[d] + 4;
    vol.assign(h->tab[d].begin() + (size_t)T_VOL * np, h->tab[d].begin() + (size_t)(T_VOL + 1) * np);
    e = cudaMemcpyAsync(h->ws + off, vol.data(), np * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "volume upload");
    off += align_up((size_t)np * sizeof(double));
  }
  {  // the device copy in the layout ptab_node_major picks; the host keeps the group-major table
    // (one table per group, ngroups of them: with three species the channels share them)
    const int G = h->P.ngroups, nu = h->ptab_nu;
    const bool nmaj = ptab_node_major(h);
    std::vector<float4> nm((size_t)G * nu);
    for (int g = 0; g < G; ++g)
      for (int i = 0; i < nu; ++i) nm[nmaj ? (size_t)i * G + g : (size_t)g * nu + i] = h->ptab[(size_t)g * nu + i];
    e = cudaMemcpyAsync(h->ws + h->off_ptab, nm.data(), nm.size() * sizeof(float4),
                        cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "Planck table upload");
  e = cudaMemcpyAsync(h->ws + h->off_gc, &h->gc, sizeof(GroupConst), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ws + h->off_vtc, &h->vtc, sizeof(VtConst), cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) {
    const std::vector<double> hr = hrows(h);
    e = cudaMemcpyAsync(h->ws + h->off_hrow, hr.data(), hr.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // hr is a local
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "group constants upload");
  if (h->layers.n > 0) {  // the layers' device copy lives in the workspace: set it in the new one
    LayerSet S = h->layers;
    S.t = h->time;
#ifdef FX_BOUNDS_CHECK
    S.status = reinterpret_cast<unsigned*>(h->ws + h->off_status);
#endif
    e = cudaMemcpyAsync(h->ws + h->off_layers, &S, sizeof(LayerSet), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "boundary layer upload");
  }
  return FX_OK;
}

fx_status fx_state_upload(fx_grid* h, const void* src, int src_precision, int src_is_device) {
  if (!h || !src) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  const int64_t n = (int64_t)h->ncell * h->NV;
  void* dst = h->ws + h->off_A;
  const int my = h->elem == 8 ? FX_FP64 : FX_FP32;  // element type of the device state
  cudaError_t e = cudaSuccess;
  if (src_precision == my) {
    e = cudaMemcpyAsync(dst, src, h->state_bytes, src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream);
    if (!src_is_device && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  } else if (!src_is_device) {
    if (my == FX_FP32) {
      std::vector<float> f((const double*)src, (const double*)src + n);
      e = cudaMemcpyAsync(dst, f.data(), n * 4, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    } else {
      std::vector<double> f((const float*)src, (const float*)src + n);
      e = cudaMemcpyAsync(dst, f.data(), n * 8, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
  } else {
    int nb = (int)((n + 255) / 256);
    if (my == FX_FP32) k_convert<double, float><<<nb, 256, 0, h->stream>>>((const double*)src, (float*)dst, n);
    else k_convert<float, double><<<nb, 256, 0, h->stream>>>((const float*)src, (double*)dst, n);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "state upload");
  return FX_OK;
}

fx_status fx_state_init_equilibrium(fx_grid* h, const double* prim, int prim_is_device) {
  if (!h || !prim) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  const int D = h->D, NP = 3 + D + (h->dg.species > 1 ? 1 : 0);
  const GroupConst* gc = reinterpret_cast<const GroupConst*>(h->ws + h->off_gc);
  // host primitives go through the second state buffer (free between steps), as many cells at a
  // time as fit: one copy per primitive row of the chunk, then the kernel for the chunk's cells
  const int64_t chunk = prim_is_device ? h->ncell
                        : std::min<int64_t>(h->ncell, (int64_t)(h->state_bytes / ((size_t)NP * sizeof(double))));
  if (chunk < 1) return fail(h, FX_ERR_UNSUPPORTED, "the state buffer cannot hold one cell's primitives");
  double* scratch = reinterpret_cast<double*>(h->ws + h->off_B);
  cudaError_t e = cudaSuccess;
  for (int64_t c0 = 0; c0 < h->ncell && e == cudaSuccess; c0 += chunk) {
    const int64_t nc = std::min<int64_t>(chunk, h->ncell - c0);
    const double* dprim = prim;
    int64_t ps = h->ncell;
    if (!prim_is_device) {
      for (int r = 0; r < NP && e == cudaSuccess; ++r)
        e = cudaMemcpyAsync(scratch + (size_t)r * nc, prim + (size_t)r * h->ncell + c0, (size_t)nc * sizeof(double),
                            cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) break;
      dprim = scratch;
      ps = nc;
    }
    const int nb = (int)((nc * (h->G + 1) + 255) / 256);
    const double* hr = h->P.geom != FX_CART ? reinterpret_cast<const double*>(h->ws + h->off_hrow) : nullptr;
    if (h->elem == 8)
      k_init_equilibrium<double><<<nb, 256, 0, h->stream>>>(dprim, c0, nc, ps, (double*)(h->ws + h->off_A), h->dg, gc, h->pk, hr);
    else
      k_init_equilibrium<float><<<nb, 256, 0, h->stream>>>(dprim, c0, nc, ps, (float*)(h->ws + h->off_A), h->dg, gc, h->pk, hr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !prim_is_device) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "equilibrium initialisation");
  return FX_OK;
}

fx_status fx_step(fx_grid* h, double dt, int nsteps) {
  if (!h) return FX_ERR_ARG;
  if (h->sticky != FX_OK) return h->sticky;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  if (!(dt > 0.0) || nsteps < 0) return fail(h, FX_ERR_ARG, "dt must be > 0 and nsteps >= 0");
  if (h->elem == 8) return enqueue_steps<double, double>(h, dt, nsteps);
  if (h->P.precision == FX_FP32_F64NEWTON) return enqueue_steps<float, double>(h, dt, nsteps);
  return enqueue_steps<float, float>(h, dt, nsteps);
}

fx_status fx_sync(fx_grid* h) {
  if (!h) return FX_ERR_ARG;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  cudaError_t e = cudaMemcpyAsync(h->h_status, h->ws + h->off_status, 6 * sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "synchronise");
  unsigned s = *h->h_status;
  if (s & ST_BOUNDS) return fail(h, FX_ERR_BOUNDS, bounds_message(h->h_status));
  if (s & ST_NONFINITE) return fail(h, FX_ERR_NONFINITE, "non-finite value in the state");
  if (s & ST_NEWTON) return fail(h, FX_ERR_NEWTON, "coupling Newton/bisection did not converge");
  if (s & ST_FLOOR) return fail(h, FX_ERR_FLOOR, "a density, pressure or radiation floor was applied");
  return h->sticky;
}

fx_status fx_conserved_totals(fx_grid* h, double out[FX_NTOTALS]) {
  if (!h || !out) return FX_ERR_ARG;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  double* part = reinterpret_cast<double*>(h->ws + h->off_tot);
  double* res = part + TOT_BLOCKS * FX_NTOTALS * 2;
  size_t off = h->off_tot + align_up((size_t)(TOT_BLOCKS * FX_NTOTALS * 2 + FX_NTOTALS) * sizeof(double));
  const double* vol[3] = {nullptr, nullptr, nullptr};
  for (int d = 0; d < h->D; ++d) {
    vol[d] = reinterpret_cast<const double*>(h->ws + off);
    off += align_up((size_t)(h->P.n[d] + 4) * sizeof(double));
  }
  for (int d = h->D; d < 3; ++d) vol[d] = vol[0];
  if (h->elem == 8)
    k_totals_partial<double><<<TOT_BLOCKS, TOT_THREADS, 0, h->stream>>>((const double*)(h->ws + h->off_A), h->dg, vol[0], vol[1], vol[2], part);
  else
    k_totals_partial<float><<<TOT_BLOCKS, TOT_THREADS, 0, h->stream>>>((const float*)(h->ws + h->off_A), h->dg, vol[0], vol[1], vol[2], part);
  k_totals_final<<<1, 32, 0, h->stream>>>(part, TOT_BLOCKS, res);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, FX_NTOTALS * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "totals");
  for (int q = h->D; q < 3; ++q) out[1 + q] = 0.0;
  return FX_OK;
}

fx_status fx_state_download(fx_grid* h, void* dst, int dst_precision, int dst_is_device) {
  if (!h || !dst) return FX_ERR_ARG;
  if (!has_ws(h)) return fail(h, FX_ERR_WORKSPACE, "no workspace bound");
  const int64_t n = (int64_t)h->ncell * h->NV;
  const void* src = h->ws + h->off_A;
  const int my = h->elem == 8 ? FX_FP64 : FX_FP32;  // element type of the device state
  cudaError_t e = cudaSuccess;
  if (dst_precision == my) {
    e = cudaMemcpyAsync(dst, src, h->state_bytes, dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream);
    if (!dst_is_device && e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  } else if (!dst_is_device) {
    if (my == FX_FP32) {
      std::vector<float> f(n);
      e = cudaMemcpyAsync(f.data(), src, n * 4, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      double* d = (double*)dst;
      for (int64_t i = 0; i < n; ++i) d[i] = f[i];
    } else {
      std::vector<double> f(n);
      e = cudaMemcpyAsync(f.data(), src, n * 8, cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      float* d = (float*)dst;
      for (int64_t i = 0; i < n; ++i) d[i] = (float)f[i];
    }
  } else {
    int nb = (int)((n + 255) / 256);
    if (my == FX_FP32) k_convert<float, double><<<nb, 256, 0, h->stream>>>((const float*)src, (double*)dst, n);
    else k_convert<double, float><<<nb, 256, 0, h->stream>>>((const double*)src, (float*)dst, n);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "state download");
  return FX_OK;
}

const char* fx_last_error(const fx_grid* h) { return h ? h->err.c_str() : "null handle"; }

void fx_clear_error(fx_grid* h) {
  if (!h) return;
  h->sticky = FX_OK;
  h->err.clear();
  if (h->ws) {
    cudaMemsetAsync(h->ws + h->off_status, 0, 64, h->stream);
    cudaStreamSynchronize(h->stream);
  }
}

fx_status fx_kernel_timing_enable(fx_grid* h, int on) {
  if (!h) return FX_ERR_ARG;
  h->timing = on != 0;
  h->nev = 0;
  return FX_OK;
}

fx_status fx_kernel_timing_read(fx_grid* h, double out[6]) {
  if (!h || !out) return FX_ERR_ARG;
  for (int q = 0; q < 6; ++q) out[q] = 0.0;
  if (h->nev == 0) return FX_OK;
  cudaError_t e = cudaEventSynchronize(h->ev[h->nev - 1]);
  if (e != cudaSuccess) return cuda_fail(h, e, "timing read");
  // the interval after the radiation/update kernel holds the velocity-term and interaction kernels
  const bool split = h->P.couple != 0 || h->P.vterms != 0;
  for (size_t i = 0; i < h->nev; i += 4) {
    float face = 0.f, stage = 0.f, inter = 0.f;
    e = cudaEventElapsedTime(&face, h->ev[i], h->ev[i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&stage, h->ev[i + 1], h->ev[i + 2]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&inter, h->ev[i + 2], h->ev[i + 3]);
    if (e != cudaSuccess) return cuda_fail(h, e, "timing read");
    out[0] += stage;
    out[1] += 1.0;
    out[2] += face;
    out[3] += 1.0;
    if (split) {
      out[4] += inter;
      out[5] += 1.0;
    }
  }
  h->nev = 0;
  return FX_OK;
}

void fx_grid_destroy(fx_grid* h) {
  if (!h) return;
  if (h->step_exec) cudaGraphExecDestroy(h->step_exec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (cudaEvent_t x : h->ev) cudaEventDestroy(x);
  if (h->h_status) cudaFreeHost(h->h_status);
  delete h;
}

// Host-side inspection of the reconstruction table of direction d (FP64 master copy):
// out receives NTAB * (n[d] + 4) doubles (entry-major).  Needs no GPU.
int fx_debug_table(const fx_grid* h, int d, double* out, size_t cap) {
  if (!h || d < 0 || d >= h->D) return -1;
  const std::vector<double>& T = h->tab[d];
  if (cap < T.size()) return (int)T.size();
  std::memcpy(out, T.data(), T.size() * sizeof(double));
  return (int)T.size();
}
int fx_debug_ntab(void) { return NTAB; }

int fx_debug_planck_table(const fx_grid* h, float* out, size_t cap, int* nu, float* u0) {
  if (!h) return -1;
  if (nu) *nu = h->ptab_nu;
  if (u0) *u0 = h->ptab_u0;
  const size_t n = h->ptab.size() * 4;
  if (out && cap >= n) std::memcpy(out, h->ptab.data(), n * sizeof(float));
  return (int)n;
}


}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Initialisation without allocation.  fx_state_init_equilibrium stages host primitives in the
// workspace's second state buffer; this variant stages them, together with the group constants,
// in a file-scope device array of fixed size that every GPU loading the library holds until the
// process exits.  Host code must not use the array's name as a device address, so each device
// resolves it once with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocBytes = (size_t)64 << 20;  // FX_NOALLOC_STAGE_BYTES in fx.h
static __device__ __align__(256) unsigned char g_noalloc_stage[kNoAllocBytes];
constexpr size_t kNoAllocGcBytes = 1024;  // GroupConst slot at the start of the array
static_assert(sizeof(GroupConst) <= kNoAllocGcBytes, "group constants do not fit their slot");
static_assert(NBUDGET == FX_NBUDGET, "budget accumulators per row and the ABI's budget count differ");
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" fx_status fx_state_init_equilibrium_noalloc(fx_grid* h, const double* prim, void* state,
                                                      int state_precision, void* cuda_stream) {
  if (!h || !prim || !state) return FX_ERR_ARG;
  if (state_precision != FX_FP64 && state_precision != FX_FP32) return fail(h, FX_ERR_ARG, "state precision must be FX_FP64 or FX_FP32");
  if (h->sticky != FX_OK) return h->sticky;
  const size_t pbytes = (size_t)(3 + h->D + (h->dg.species > 1 ? 1 : 0)) * h->ncell * sizeof(double);
  // curvilinear grids: the scale-factor rows T_HA, T_HB of each direction, staged after the
  // primitives straight from the handle's tables (nothing is allocated)
  size_t hbytes = 0;
  if (h->P.geom != FX_CART)
    for (int d = 0; d < h->D; ++d) hbytes += 2 * (size_t)(h->P.n[d] + 4) * sizeof(double);
  if (pbytes + hbytes > kNoAllocBytes - kNoAllocGcBytes)
    return fail(h, FX_ERR_UNSUPPORTED,
                "fx_state_init_equilibrium_noalloc: the primitives (" + std::to_string(pbytes) +
                    " bytes) exceed its fixed device staging array (" +
                    std::to_string(kNoAllocBytes - kNoAllocGcBytes) + " bytes)");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(h, FX_ERR_UNSUPPORTED, "device ordinal beyond the supported range");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      // once per device, with that device current
      e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_stage);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return cuda_fail(h, e, "cudaGetSymbolAddress of the staging array");
      }
    }
    base = g_noalloc_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  unsigned char* stage = static_cast<unsigned char*>(base);
  e = cudaMemcpyAsync(stage, &h->gc, sizeof(GroupConst), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(stage + kNoAllocGcBytes, prim, pbytes, cudaMemcpyHostToDevice, s);
  if (hbytes) {
    size_t off = kNoAllocGcBytes + pbytes;
    for (int d = 0; d < h->D && e == cudaSuccess; ++d) {
      const size_t np = (size_t)h->P.n[d] + 4;
      for (int row : {T_HA, T_HB}) {
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(stage + off, h->tab[d].data() + row * np, np * sizeof(double), cudaMemcpyHostToDevice, s);
        off += np * sizeof(double);
      }
    }
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "staging copy");
  const int64_t nt = h->ncell * (h->G + 1);
  const int nb = (int)((nt + 255) / 256);
  const GroupConst* gc = reinterpret_cast<const GroupConst*>(stage);
  const double* dprim = reinterpret_cast<const double*>(stage + kNoAllocGcBytes);
  const double* dh = hbytes ? reinterpret_cast<const double*>(stage + kNoAllocGcBytes + pbytes) : nullptr;
  if (state_precision == FX_FP64)
    k_init_equilibrium<double><<<nb, 256, 0, s>>>(dprim, 0, h->ncell, h->ncell, static_cast<double*>(state),
                                                  h->dg, gc, h->pk, dh);
  else
    k_init_equilibrium<float><<<nb, 256, 0, s>>>(dprim, 0, h->ncell, h->ncell, static_cast<float*>(state),
                                                 h->dg, gc, h->pk, dh);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "equilibrium initialisation (no-alloc)");
  return FX_OK;
}

