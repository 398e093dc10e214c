// Float-float arithmetic and the control logic of the refinement loop
// (device code shared by the single-grid and the batched solvers).
#pragma once
#include <math.h>

#include "launch.h"

namespace npmg {

__device__ __forceinline__ double pow2_floor(double v) {
  if (!(v > 0.0) || !isfinite(v)) return 1.0;
  int e;
  frexp(v, &e);
  return ldexp(1.0, e - 1);
}

// ---------------------------------------------------------------------------
// Float-float arithmetic (Dekker 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2):
// a value is hi + lo with |lo| <= ulp(hi)/2, about 48 significant bits.
// GB300 runs float64 at 1/64 of the float32 rate, so the refinement
// residual uses these float32 sequences instead.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
// (a.hi + a.lo) * (w.hi + w.lo), dropping the lo * lo term.
__device__ __forceinline__ ff ff_mul(ff a, ff w) {
  const float p = a.hi * w.hi;
  float e = fmaf(a.hi, w.hi, -p);
  e = fmaf(a.hi, w.lo, e);
  e = fmaf(a.lo, w.hi, e);
  return quick_two_sum(p, e);
}

// Refinement step decision from ||r||^2 (scaled units; divided by c^2 to
// get unscaled units): converged, diverged, out of steps or stalled;
// otherwise the tolerance of the next inner solve.
__device__ __forceinline__ void outer_decide(SolveState* st, double tot, double c2, double sig_new, bool update) {
  const double bn2 = st->bnorm2;
  const double rel = bn2 > 0.0 ? sqrt(tot / (c2 * bn2)) : 0.0;
  const double prev = st->relres;
  if (update) st->outer += 1;
  const int o = st->outer;
  if (o < kHistory) st->hist[o] = rel;
  if (!update) st->relres0 = rel;
  st->relres = rel;
  st->sigma = sig_new;
  bool done = false;
  if (bn2 == 0.0 || rel <= st->tol) {
    st->status = MG_OK;
    done = true;
  } else if (!isfinite(rel) || rel > 1e3 * fmax(st->relres0, 1.0) || st->status == MG_DIVERGED) {
    st->status = MG_DIVERGED;
    done = true;
  } else if (o >= st->max_outer) {
    st->status = MG_NOT_CONVERGED;
    done = true;
  } else {
    if (update && rel > 0.9 * prev) st->stall += 1;
    if (st->stall >= 3) {
      st->status = MG_NOT_CONVERGED;
      done = true;
    }
  }
  st->outer_done = done ? 1 : 0;
  if (!done) {
    st->eta = fmax(0.5 * st->tol / rel, st->inner_floor);
    st->r0norm2 = tot / (sig_new * sig_new);
    st->inner_done = 0;
    st->it = 0;
    st->first = 1;
  } else {
    st->inner_done = 1;
  }
}

// CG step bookkeeping from ||r||^2: iteration counts and convergence.
__device__ __forceinline__ void inner_decide(SolveState* st, double tot) {
  st->rnorm2 = tot;
  st->it += 1;
  st->iters_total += 1;
  st->first = 0;
  if (!isfinite(tot) || tot > 1e12 * st->r0norm2) {
    st->status = MG_DIVERGED;
    st->inner_done = 1;
    st->outer_done = 1;
  } else if (tot <= st->eta * st->eta * st->r0norm2 || st->it >= st->max_inner) {
    st->inner_done = 1;
  }
}

// Solve start: parameters, ||b||^2 and the first scale sigma = c rms(b).
__device__ __forceinline__ void init_state(SolveState* st, const SolveParams& prm, double bnorm2, double c) {
  st->tol = prm.tol;
  st->inner_floor = prm.inner_floor;
  st->max_inner = prm.max_inner;
  st->max_outer = prm.max_outer;
  st->krylov = prm.krylov;
  st->n_fluid = prm.n_fluid;
  st->bnorm2 = bnorm2;
  st->relres = 1.0;
  st->relres0 = 1.0;
  st->sigma = bnorm2 > 0.0 ? pow2_floor(c * sqrt(bnorm2 / (double)prm.n_fluid)) : 1.0;
  st->eta = 1.0;
  st->outer = 0;
  st->outer_done = 0;
  st->status = MG_OK;
  st->stall = 0;
  for (int k = 0; k < kHistory; ++k) st->hist[k] = 0.0;
  st->inner_done = 1;
  st->it = 0;
  st->iters_total = 0;
  st->first = 1;
  st->r0norm2 = 0.0;
  st->rz = st->rz_old = st->alpha = st->beta = st->rnorm2 = st->pAp = 0.0;
}

}  // namespace npmg
