// Boundary layers (the double Mach reflection of Sec. 8.4 and other fixed or time-dependent
// boundaries): boxes of grid cells overwritten before each stage and after each step, with one of
// two states split by a moving straight front (x - x0 - (y - y0) cot(alpha) - s t <= 0: state A)
// or with the mirror image of the interior across a plane (a reflecting wall on part of a side,
// normal momentum and flux negated).  The boxes do not overlap and no mirror reads a box, so the
// layers of one launch are independent.
#pragma once
#include "fx_check.cuh"
#include "fx_types.h"

namespace fx {

constexpr int MAX_LAYERS = 8;
constexpr int LAYER_THREADS = 256;

struct LayerDev {
  int kind;  // 0 front, 1 mirror
  int d, m;  // mirror: cell i along d takes cell 2m - 1 - i
  int lo[3], hi[3];
  double x0, y0, cot, speed;
  double UA[5 + MAXG], UB[5 + MAXG];  // front: conserved gas (2 + D values), then E_g (F = 0)
};
struct LayerSet {
  int n;
  double x_lo[3], dx[3];
  LayerDev L[MAX_LAYERS];
  double t;  // time at the start of the current step (device copy: advanced by layer_advance)
#ifdef FX_BOUNDS_CHECK
  unsigned* status;  // status word and state elements for the index checks of the debug build
  int64_t n_state;
#endif
};

// Grid row y = layer; the cells of its box strided over the row's blocks.  The layers are set at
// time S->t + toff (toff = 0 for the stage-1 input, dt for the stage-2 input and the result), so
// that a step's launches do not change from step to step (a captured graph replays them).
template <class R>
__global__ void __launch_bounds__(LAYER_THREADS) layer_kernel(const LayerSet* S, R* U, const DevGrid g, double toff) {
  const int q = blockIdx.y;
  if (q >= S->n) return;
  const double t = S->t + toff;
  const LayerDev& L = S->L[q];
  const int D = g.D, G = g.G, NG = 2 + D;
  const int bx = L.hi[0] - L.lo[0], by = L.hi[1] - L.lo[1], bz = L.hi[2] - L.lo[2];
  const int64_t nb = (int64_t)bx * by * bz, ncell = g.ncell;
  for (int64_t e = (int64_t)blockIdx.x * LAYER_THREADS + threadIdx.x; e < nb;
       e += (int64_t)gridDim.x * LAYER_THREADS) {
    const int c3[3] = {L.lo[0] + (int)(e % bx), L.lo[1] + (int)((e / bx) % by), L.lo[2] + (int)(e / ((int64_t)bx * by))};
    const int64_t c = ((int64_t)c3[2] * g.n[1] + c3[1]) * g.n[0] + c3[0];
    if (L.kind == 1) {
      int s3[3] = {c3[0], c3[1], c3[2]};
      s3[L.d] = 2 * L.m - 1 - c3[L.d];
      const int64_t cs = ((int64_t)s3[2] * g.n[1] + s3[1]) * g.n[0] + s3[0];
      for (int v = 0; v < NG; ++v) {
        const R x = U[FXI_AT(S->status, v * ncell + cs, S->n_state)];
        U[FXI_AT(S->status, v * ncell + c, S->n_state)] = v == 1 + L.d ? -x : x;
      }
      for (int v = 0; v <= D; ++v)
        for (int k = 0; k < G; ++k) {
          const R x = U[FXI_AT(S->status, NG * ncell + (v * ncell + cs) * G + k, S->n_state)];
          U[FXI_AT(S->status, NG * ncell + (v * ncell + c) * G + k, S->n_state)] = v == 1 + L.d ? -x : x;
        }
      continue;
    }
    // cell centres x_lo + i dx + dx/2 and the front, rounded operation by operation (no FMA
    // contraction: the side of the front each cell takes is decided as on the host)
    const double xc = __dadd_rn(__dadd_rn(S->x_lo[0], __dmul_rn((double)c3[0], S->dx[0])), __dmul_rn(0.5, S->dx[0]));
    const double yc = D > 1 ? __dadd_rn(__dadd_rn(S->x_lo[1], __dmul_rn((double)c3[1], S->dx[1])), __dmul_rn(0.5, S->dx[1])) : 0.0;
    const double f = __dsub_rn(__dsub_rn(__dsub_rn(xc, L.x0), __dmul_rn(__dsub_rn(yc, L.y0), L.cot)), __dmul_rn(L.speed, t));
    const double* W = f <= 0.0 ? L.UA : L.UB;
    for (int v = 0; v < NG; ++v) U[FXI_AT(S->status, v * ncell + c, S->n_state)] = (R)W[v];
    for (int k = 0; k < G; ++k) {
      U[FXI_AT(S->status, NG * ncell + c * G + k, S->n_state)] = (R)W[NG + k];
      for (int v = 1; v <= D; ++v) U[FXI_AT(S->status, NG * ncell + (v * ncell + c) * G + k, S->n_state)] = R(0);
    }
  }
}

// The end of a step: the layers' time advances by dt (one thread, after the step's last layer
// launch on the same stream).
__global__ void layer_advance(LayerSet* S, double dt) {
  if (threadIdx.x == 0 && blockIdx.x == 0) S->t = S->t + dt;
}

}  // namespace fx
