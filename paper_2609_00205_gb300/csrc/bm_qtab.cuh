// max|u| accumulation and the quantiser table (Sec. III-C error budget),
// shared by the max|u| pass of a compress call and the batched forward
// kernel, which computes both inside its persistent launch.
#pragma once

#include "bm_common.cuh"

namespace bm {

template <typename T>
__device__ __forceinline__ void maxabs_acc(T x, T& m, bool& bad) {
  const T v = fabs(x);
  bad |= !(v < T(INFINITY));  // NaN or infinity: the stream will be raw
  m = v > m ? v : m;          // NaN never compares greater: ignored; infinity kept
}

// Quantiser widths of every (tier, level), in IEEE double arithmetic without
// contraction: tau' = tau - margin, margin = kappa eps (N+1) max|u|;
// q_level = 2 tau'/((N+1) A_level), q_coarsest = 2 tau_g'/(N+1).
struct QtabArgs {
  int enabled;
  const double* tiers;  // relative or absolute, ascending
  int ntiers, rel, K, M, R;
  double A[24];
  double kappa, eps;
  double* qd;           // [ntiers*K + M + 1]
  void* rq;             // same count, field dtype
  int f64;
  uint8_t* out;         // stream (tiers + qtab sections) or null
  unsigned long long off_tiers, off_qtab;
  Scalars* sc;
};

__device__ inline void qtab_compute(const QtabArgs& a) {
  const double max_abs = a.f64 ? __longlong_as_double((long long)a.sc->maxabs_bits)
                               : (double)__uint_as_float((unsigned)a.sc->maxabs_bits);
  const int N = a.R * a.K + a.M;
  const double t = (double)(N + 1);
  const double margin = __dmul_rn(__dmul_rn(__dmul_rn(a.kappa, a.eps), t), max_abs);
  bool raw = !isfinite(max_abs);
  double taug = INFINITY;
  const int nq = a.ntiers * a.K + a.M + 1;
  for (int i = 0; i < a.ntiers; ++i) {
    const double tau = a.rel ? __dmul_rn(a.tiers[i], max_abs) : a.tiers[i];
    if (a.out) reinterpret_cast<double*>(a.out + a.off_tiers)[i] = tau;
    const double taup = __dsub_rn(tau, margin);
    if (!(taup > __dmul_rn(0.5, tau))) raw = true;
    taug = fmin(taug, taup);
    for (int l = 0; l < a.K; ++l)
      a.qd[i * a.K + l] = __dmul_rn(2.0, __ddiv_rn(taup, __dmul_rn(t, a.A[l])));
  }
  for (int l = 0; l < a.M; ++l) a.qd[a.ntiers * a.K + l] = __dmul_rn(2.0, __ddiv_rn(taug, __dmul_rn(t, a.A[a.K + l])));
  a.qd[nq - 1] = __dmul_rn(2.0, __ddiv_rn(taug, t));
  for (int i = 0; i < nq; ++i) {
    const double r = __ddiv_rn(1.0, a.qd[i]);
    if (a.f64) reinterpret_cast<double*>(a.rq)[i] = r;
    else reinterpret_cast<float*>(a.rq)[i] = __double2float_rn(r);
    if (a.out) reinterpret_cast<double*>(a.out + a.off_qtab)[i] = a.qd[i];
  }
  a.sc->max_abs = max_abs;
  a.sc->margin = margin;
  if (raw) atomicOr(&a.sc->status, ST_RAW);
}

}  // namespace bm
