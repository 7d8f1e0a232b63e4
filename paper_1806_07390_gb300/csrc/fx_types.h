// Internal types shared by the host driver and the kernels of the stage update.
#pragma once
#include <stddef.h>
#include <stdint.h>

namespace fx {

constexpr int MAXG = 32;          // groups per cell handled by one lane segment
constexpr int NPLANCK_LO = 27;    // FP64 Bernoulli-series terms (x < XSPLIT, error < 1e-17)
constexpr int NPLANCK_LO32 = 13;  // FP32 Bernoulli-series terms (error < 1e-8)
constexpr int NPLANCK_UP = 48;    // cap of the FP64 exponential series (x >= XSPLIT: 14 terms)
constexpr double XSPLIT = 3.0;    // lower/upper Planck series switch
constexpr int NBUDGET = 9;        // budget accumulators per row (see StageArgs::budget)
constexpr int BUDGET_SLOTS = 64;  // rows of budget accumulators that blocks add to (summed when read)
constexpr int PTAB_PER_OCT = 32;  // FP32 Planck band tables: nodes per octave of T
constexpr double PTAB_XMAX = 88.0;   // below T = eps_min/88 every band underflows in FP32
constexpr double PTAB_XMIN = 6.103515625e-05;  // 2^-14: above T = eps_max/2^-14, series in x

// Status bits raised by kernels (atomicOr into the workspace status word).
enum : unsigned {
  ST_NEWTON = 1u,     // Newton and bisection did not converge in some cell
  ST_FLOOR = 2u,      // a floor was applied
  ST_NONFINITE = 4u,  // a non-finite value was produced
  ST_BOUNDS = 8u,     // an index fell outside its buffer (index checks of the debug build)
};

// Kernel-side description of the grid (passed by value to every launch).
struct DevGrid {
  int D, G;
  int n[3];          // cells per direction (1 for inactive directions)
  int bc_lo[3], bc_hi[3];
  int geom;
  int64_t ncell;
  double gamma, c, a_rad;
  double kappa0, sigma0;
  int kap_rho_h, kap_T_h;  // opacity exponents in halves
  double rho_floor, p_floor, E_floor;
  int newton_maxit, bisect_maxit;
  double newton_rtol;
  int couple;
  int rad_order;  // radiation reconstruction: 1 linear with the MC limiter, 2 the gas's parabola
  int riemann;        // gas solver: 0 HLLC, 1 HLLE, 2 local Lax-Friedrichs
  double shock_guard; // carbuncle guard pressure-jump threshold (0: off)
  int vterms;         // velocity-dependent radiation terms on
  double inv_dx[3];   // 1 / cell width per direction (in x, the coordinate)
  int species;        // 1, or 3: G = 3 Gs channels, composition rho Y_e, (T, Y_e) interaction
  int Gs;             // groups per species (channel k is group k % Gs of species k / Gs)
  double xi0;         // lepton number per unit energy of the nu_e / anti-nu_e channels
};

}  // namespace fx
