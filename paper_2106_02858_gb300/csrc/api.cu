// C ABI of libcmcg: handle life cycle, period sweeps and the CMCG driver.
//
// Sweeps (Section 4.1.2, Algorithms rk2 / rk4).  Every stage is one launch of
// the stage kernel over all tetrahedra; the state being propagated lives in
// the handle's work vector Uw.
//   * source-free sweeps (P_w, P*_w) use the nested (Horner) form of the RK
//     polynomial, v <- U + (dt / k) B v for k = s, ..., 1, which is the same
//     polynomial sum_k (dt B)^k / k! as Algorithms rk2 / rk4 for a linear
//     autonomous system and differs from them only by rounding;
//   * sweeps with the source (P_{psi,w}, F_{psi,w}) run Algorithms rk2 / rk4 as
//     printed, with Phi(t, U) evaluated at the stage times; the filter is
//     accumulated on the fly at the first stage of every step and once more at
//     t_M (Eq. filtering_RK2 / filtering_RK4, each with the 2/T of Eq. filter).
// CMCG (Section 2.2, Algorithms init / grad / cmcg) runs in residual form from
// U0 = 0: G = P_psi 0, G* = G - P* G, R = D = G*, then per iteration
// W_T = P D - D, A = P* W_T - W_T, alpha = |R|^2 / (D, A), U0 += alpha D,
// R -= alpha A, beta = |R_new|^2 / |R|^2, D = R + beta D; the scalars are FP64
// and stay on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <new>

#include "common.h"

using namespace cmcg;

struct cmcg_handle {
  int device = 0;
  cudaStream_t stream = nullptr;
  HostLayout L;
  int q = 1, np = 4, prec = CMCG_FP64, integrator = 2;
  double omega = 0, T = 0, dt = 0;
  int M = 0;
  int64_t nt = 0, nti = 0, nvec = 0, njvec = 0;
  size_t rsize = 8;
  // device memory
  void *gvol = nullptr, *gface = nullptr;
  int32_t* nbr = nullptr;
  double* wdot = nullptr;
  int32_t* e_of_i = nullptr;
  double* inv_eps = nullptr;
  void *Uw = nullptr, *vA = nullptr, *vB = nullptr, *ACC = nullptr, *Fre = nullptr, *Fim = nullptr;
  void *Jre = nullptr, *Jim = nullptr;
  void *U0 = nullptr, *Rv = nullptr, *D = nullptr, *A = nullptr, *WT = nullptr;
  double* partials = nullptr;
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned
  double *ext0 = nullptr, *ext1 = nullptr, *ext2 = nullptr, *ext3 = nullptr;
  int64_t launches = 0;
  size_t bytes = 0;
  int variant = 0;     // occupancy variant of the per-stage kernel
  int packed_minb = 0; // > 0 (FP32): every stage runs on the packed two-tetrahedra-per-lane kernel
  int nsm = 0;
  double tune_us[8];
  std::vector<std::complex<double>> fa, fb;  // filter weights per step 0..M
  // sweep profiling
  bool prof = false;
  struct SweepEv {
    cudaEvent_t a, b;
    bool source;
    int64_t stages;
  };
  std::vector<SweepEv> prof_ev;
  size_t prof_used = 0;
  double prof_ms[2] = {0, 0};
  int64_t prof_stages[2] = {0, 0};
};

namespace {

std::mutex g_const_mutex;
bool g_const_uploaded[64][4] = {};

int cuda_fail(cudaError_t e) {
  if (e == cudaErrorMemoryAllocation) return CMCG_ERR_OUT_OF_MEMORY;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver || e == cudaErrorInvalidDevice)
    return CMCG_ERR_NO_DEVICE;
  return CMCG_ERR_CUDA;
}

#define CK(expr)                               \
  do {                                         \
    cudaError_t e_ = (expr);                   \
    if (e_ != cudaSuccess) return cuda_fail(e_); \
  } while (0)

int ensure_constants(int device, int q) {
  std::lock_guard<std::mutex> lk(g_const_mutex);
  if (device < 0 || device >= 64) return CMCG_ERR_INVALID_ARG;
  if (g_const_uploaded[device][q]) return CMCG_OK;
  const RefMats& rm = ref_mats(q);
  if (q == 1) upload_constants<1>(rm);
  else if (q == 2) upload_constants<2>(rm);
  else upload_constants<3>(rm);
  upload_dot_mass(q, rm.M.data());
  CK(cudaGetLastError());
  g_const_uploaded[device][q] = true;
  return CMCG_OK;
}

// Filter weights a_m, b_m (m = 0..M) of F += a_m U_m + b_m Phi_m, including 2/T.
// The Hermite moments I_k(theta) = int_0^1 s^k e^{-i theta s} ds are computed
// with a 24-point Gauss-Legendre rule (exact to rounding for the small theta
// = w dt of a stable step).
void filter_weights(cmcg_handle* h) {
  const int M = h->M;
  const double dt = h->dt, w = h->omega, c = 2.0 / h->T;
  h->fa.assign(M + 1, 0.0);
  h->fb.assign(M + 1, 0.0);
  using cd = std::complex<double>;
  if (h->integrator == 2) {
    for (int m = 0; m <= M; ++m) {
      const double wt = (m == 0 || m == M) ? 0.5 : 1.0;
      h->fa[m] = c * dt * wt * std::exp(cd(0, -w * m * dt));
    }
    return;
  }
  std::vector<double> gx, gw;
  gauss_legendre01(24, gx, gw);
  const double th = w * dt;
  cd I[4] = {0, 0, 0, 0};
  for (size_t p = 0; p < gx.size(); ++p) {
    const cd e = std::exp(cd(0, -th * gx[p]));
    double sk = 1;
    for (int k = 0; k < 4; ++k) {
      I[k] += gw[p] * sk * e;
      sk *= gx[p];
    }
  }
  // Hermite cubics on s in [0,1]: p00 = 1 - 3s^2 + 2s^3, p01 = 3s^2 - 2s^3,
  // p10 = dt (s - 2s^2 + s^3), p11 = dt (s^3 - s^2); each interval [t_{m-1}, t_m]
  // carries the factor dt e^{-i w t_{m-1}}.
  const cd x00 = I[0] - 3.0 * I[2] + 2.0 * I[3], x01 = 3.0 * I[2] - 2.0 * I[3];
  const cd x10 = dt * (I[1] - 2.0 * I[2] + I[3]), x11 = dt * (I[3] - I[2]);
  for (int m = 1; m <= M; ++m) {
    const cd e = dt * std::exp(cd(0, -w * (m - 1) * dt));
    h->fa[m - 1] += c * e * x00;
    h->fa[m] += c * e * x01;
    h->fb[m - 1] += c * e * x10;
    h->fb[m] += c * e * x11;
  }
}

template <typename R>
void stage(cmcg_handle* h, StageArgs<R>& a) {
  a.gvol = (const R*)h->gvol;
  a.gface = (const R*)h->gface;
  a.nbr = h->nbr;
  a.nti = h->nti;
  if constexpr (sizeof(R) == 4) {
    if (h->packed_minb > 0) {
      if (h->q == 1) launch_stage_packed<1>(a, h->stream, h->packed_minb);
      else if (h->q == 2) launch_stage_packed<2>(a, h->stream, h->packed_minb);
      else launch_stage_packed<3>(a, h->stream, h->packed_minb);
      h->launches++;
      return;
    }
  }
  if (h->q == 1) launch_stage<1, R>(a, h->stream, h->variant);
  else if (h->q == 2) launch_stage<2, R>(a, h->stream, h->variant);
  else launch_stage<3, R>(a, h->stream, h->variant);
  h->launches++;
}

template <typename R>
StageArgs<R> blank() {
  StageArgs<R> a;
  std::memset(&a, 0, sizeof(a));
  a.sH = R(1);
  return a;
}

// Sweep profiling: events around a sweep, collected lazily.
cmcg_handle::SweepEv* prof_begin(cmcg_handle* h, bool source) {
  if (!h->prof) return nullptr;
  if (h->prof_used == h->prof_ev.size()) {
    cmcg_handle::SweepEv e{};
    if (cudaEventCreate(&e.a) != cudaSuccess || cudaEventCreate(&e.b) != cudaSuccess) return nullptr;
    h->prof_ev.push_back(e);
  }
  cmcg_handle::SweepEv* e = &h->prof_ev[h->prof_used++];
  e->source = source;
  e->stages = h->launches;
  cudaEventRecord(e->a, h->stream);
  return e;
}
void prof_end(cmcg_handle* h, cmcg_handle::SweepEv* e) {
  if (!e) return;
  cudaEventRecord(e->b, h->stream);
  e->stages = h->launches - e->stages;
}
// Folds recorded sweeps into the totals (waits for their events).
void prof_collect(cmcg_handle* h) {
  for (size_t i = 0; i < h->prof_used; ++i) {
    cmcg_handle::SweepEv& e = h->prof_ev[i];
    cudaEventSynchronize(e.b);
    float ms = 0;
    cudaEventElapsedTime(&ms, e.a, e.b);
    h->prof_ms[e.source ? 1 : 0] += ms;
    h->prof_stages[e.source ? 1 : 0] += e.stages;
  }
  h->prof_used = 0;
}

// Source-free sweep of Uw in place (nested RK form); adjoint flips the magnetic sign.
template <typename R>
void sweep_free(cmcg_handle* h, bool adjoint) {
  cmcg_handle::SweepEv* pe = prof_begin(h, false);
  R* Uw = (R*)h->Uw;
  R* v[2] = {(R*)h->vA, (R*)h->vB};
  const int s = h->integrator;
  for (int m = 0; m < h->M; ++m) {
    const R* vin = Uw;
    int pp = 0;
    for (int k = s; k >= 1; --k) {
      StageArgs<R> a = blank<R>();
      a.vin = vin;
      a.base = Uw;
      a.out = (k == 1) ? Uw : v[pp];
      a.c_out = R(h->dt / k);
      a.sH = adjoint ? R(-1) : R(1);
      stage<R>(h, a);
      vin = a.out;
      pp ^= 1;
    }
  }
  prof_end(h, pe);
}

// Sweep with source (Algorithms rk2 / rk4 as printed) of Uw in place; optional on-the-fly filter.
template <typename R>
void sweep_source(cmcg_handle* h, bool with_source, bool filter) {
  cmcg_handle::SweepEv* pe = prof_begin(h, true);
  R* Uw = (R*)h->Uw;
  R* vA = (R*)h->vA;
  R* vB = (R*)h->vB;
  R* ACC = (R*)h->ACC;
  const double dt = h->dt, w = h->omega;
  auto src = [&](StageArgs<R>& a, double t) {
    if (!with_source) return;
    a.jre = (const R*)h->Jre;
    a.jim = (const R*)h->Jim;
    a.s_cos = R(std::cos(w * t));
    a.s_sin = R(std::sin(w * t));
  };
  auto filt = [&](StageArgs<R>& a, int m) {
    if (!filter) return;
    a.fre = (R*)h->Fre;
    a.fim = (R*)h->Fim;
    a.fa_re = R(h->fa[m].real());
    a.fa_im = R(h->fa[m].imag());
    a.fb_re = R(h->fb[m].real());
    a.fb_im = R(h->fb[m].imag());
  };
  for (int m = 0; m < h->M; ++m) {
    const double t = m * dt;
    if (h->integrator == 2) {
      StageArgs<R> a = blank<R>();
      a.vin = Uw; a.base = Uw; a.out = vA; a.c_out = R(dt / 2);
      src(a, t);
      filt(a, m);
      stage<R>(h, a);
      StageArgs<R> b = blank<R>();
      b.vin = vA; b.base = Uw; b.out = Uw; b.c_out = R(dt);
      src(b, t + dt / 2);
      stage<R>(h, b);
    } else {
      StageArgs<R> a = blank<R>();
      a.vin = Uw; a.base = Uw; a.out = vA; a.c_out = R(dt / 2);
      a.acc_in = Uw; a.acc_out = ACC; a.c_acc = R(dt / 6);
      src(a, t);
      filt(a, m);
      stage<R>(h, a);
      StageArgs<R> b = blank<R>();
      b.vin = vA; b.base = Uw; b.out = vB; b.c_out = R(dt / 2);
      b.acc_in = ACC; b.acc_out = ACC; b.c_acc = R(dt / 3);
      src(b, t + dt / 2);
      stage<R>(h, b);
      StageArgs<R> c = blank<R>();
      c.vin = vB; c.base = Uw; c.out = vA; c.c_out = R(dt);
      c.acc_in = ACC; c.acc_out = ACC; c.c_acc = R(dt / 3);
      src(c, t + dt / 2);
      stage<R>(h, c);
      StageArgs<R> d = blank<R>();
      d.vin = vA; d.base = ACC; d.out = Uw; d.c_out = R(dt / 6);
      src(d, t + dt);
      stage<R>(h, d);
    }
  }
  if (filter) {  // the t_M term: F += a_M U_M + b_M Phi(t_M, U_M)
    StageArgs<R> a = blank<R>();
    a.vin = Uw;
    src(a, h->M * dt);
    filt(a, h->M);
    stage<R>(h, a);
  }
  prof_end(h, pe);
}

// Times the stage-kernel forms on this mesh with a nested source-free stage on
// zero fields (3 warm-up + 12 timed launches each): the scalar kernel at each
// occupancy variant and, in FP32, the packed kernel; keeps the fastest.
// tune_us[0..2]: scalar variants, tune_us[3]: packed.
template <typename R>
int autotune(cmcg_handle* h, int nvariants) {
  for (double& x : h->tune_us) x = -1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaMemsetAsync(h->Uw, 0, h->nvec * h->rsize, h->stream));
  const int64_t launches0 = h->launches;
  auto time_one = [&](double* us) -> int {
    auto run = [&](int n) {
      for (int k = 0; k < n; ++k) {
        StageArgs<R> a = blank<R>();
        a.vin = (const R*)h->Uw;
        a.base = (const R*)h->vB;
        a.out = (R*)h->vA;
        a.c_out = R(h->dt);
        stage<R>(h, a);
      }
    };
    run(1);
    if (cudaGetLastError() != cudaSuccess) {  // launch rejected (configuration): form unavailable
      *us = -1;
      return CMCG_OK;
    }
    run(2);
    CK(cudaEventRecord(e0, h->stream));
    run(12);
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaGetLastError());
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    *us = 1e3 * ms / 12;
    return CMCG_OK;
  };
  CK(cudaMemsetAsync(h->vB, 0, h->nvec * h->rsize, h->stream));
  double best = 1e300;
  int bestv = 0;
  h->packed_minb = 0;
  for (int v = 0; v < nvariants; ++v) {
    h->variant = v;
    double us;
    int rc = time_one(&us);
    if (rc) return rc;
    h->tune_us[v] = us;
    if (us >= 0 && us < best) {
      best = us;
      bestv = v;
    }
  }
  h->variant = bestv;
  if (sizeof(R) == 4) {
    h->packed_minb = 2;
    double us;
    int rc = time_one(&us);
    if (rc) return rc;
    h->tune_us[3] = us;
    if (!(us >= 0 && us < best)) h->packed_minb = 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->launches = launches0;
  CK(cudaGetLastError());
  return CMCG_OK;
}

template <typename R>
void to_int(cmcg_handle* h, const double* ext, int ncomp_ext, R* in, int ncomp_in, int c_in0, int cnt,
            const double* per_tet) {
  launch_to_internal<R>(ext, ncomp_ext, 0, in, ncomp_in, c_in0, cnt, h->e_of_i, h->nti, h->np, 1.0, per_tet, h->stream);
  h->launches++;
}
template <typename R>
void to_ext(cmcg_handle* h, const R* in, int ncomp_in, int c_in0, double* ext, int ncomp_ext, int cnt) {
  launch_to_external<R>(in, ncomp_in, c_in0, ext, ncomp_ext, 0, cnt, h->e_of_i, h->nti, h->np, h->stream);
  h->launches++;
}
template <typename R>
void lincomb(cmcg_handle* h, void* o1, void* o2, void* o3, double a, const void* x, double b, const void* y) {
  launch_lincomb3<R>((R*)o1, (R*)o2, (R*)o3, a, (const R*)x, b, (const R*)y, h->nvec, h->stream);
  h->launches++;
}

template <typename R>
int set_source(cmcg_handle* h, const double* j_re, const double* j_im) {
  to_int<R>(h, j_re, 3, (R*)h->Jre, 3, 0, 3, h->inv_eps);
  if (j_im) to_int<R>(h, j_im, 3, (R*)h->Jim, 3, 0, 3, h->inv_eps);
  else CK(cudaMemsetAsync(h->Jim, 0, h->njvec * h->rsize, h->stream));
  return CMCG_OK;
}

// Device-pointer period sweeps.
template <typename R>
int forward_dev(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT, double* fre,
                double* fim) {
  to_int<R>(h, u0, 6, (R*)h->Uw, 6, 0, 6, nullptr);
  const bool filter = fre && fim;
  if (j_re) {
    int rc = set_source<R>(h, j_re, j_im);
    if (rc) return rc;
  }
  if (filter) {
    CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
    CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
  }
  if (j_re || filter) sweep_source<R>(h, j_re != nullptr, filter);
  else sweep_free<R>(h, false);
  if (uT) to_ext<R>(h, (const R*)h->Uw, 6, 0, uT, 6, 6);
  if (filter) {
    to_ext<R>(h, (const R*)h->Fre, 6, 0, fre, 6, 6);
    to_ext<R>(h, (const R*)h->Fim, 6, 0, fim, 6, 6);
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

template <typename R>
int adjoint_dev(cmcg_handle* h, const double* wT, double* w0) {
  to_int<R>(h, wT, 6, (R*)h->Uw, 6, 0, 6, nullptr);
  sweep_free<R>(h, true);
  to_ext<R>(h, (const R*)h->Uw, 6, 0, w0, 6, 6);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

template <typename R>
int apply_dev(cmcg_handle* h, double t, const double* u, const double* j_re, const double* j_im, int adjoint,
              double* out) {
  to_int<R>(h, u, 6, (R*)h->Uw, 6, 0, 6, nullptr);
  CK(cudaMemsetAsync(h->vB, 0, h->nvec * h->rsize, h->stream));
  StageArgs<R> a = blank<R>();
  a.vin = (const R*)h->Uw;
  a.base = (const R*)h->vB;
  a.out = (R*)h->vA;
  a.c_out = R(1);
  a.sH = adjoint ? R(-1) : R(1);
  if (j_re && !adjoint) {
    int rc = set_source<R>(h, j_re, j_im);
    if (rc) return rc;
    a.jre = (const R*)h->Jre;
    a.jim = (const R*)h->Jim;
    a.s_cos = R(std::cos(h->omega * t));
    a.s_sin = R(std::sin(h->omega * t));
  }
  stage<R>(h, a);
  to_ext<R>(h, (const R*)h->vA, 6, 0, out, 6, 6);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

template <typename R>
int inner_dev(cmcg_handle* h, const double* u, const double* v, double* out) {
  to_int<R>(h, u, 6, (R*)h->Uw, 6, 0, 6, nullptr);
  to_int<R>(h, v, 6, (R*)h->vA, 6, 0, 6, nullptr);
  launch_dot<R>(h->q, (const R*)h->Uw, (const R*)h->vA, h->wdot, h->partials, h->nti, h->stream);
  launch_finalize(h->partials, dot_blocks(h->nti), h->sc, 3, h->stream);
  h->launches += 2;
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->sc_host->rr_new;
  return CMCG_OK;
}

template <typename R>
int read_scalars(cmcg_handle* h) {
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

template <typename R>
int solve_dev(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
              double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, h->stream));
  const int nb = dot_blocks(h->nti);
  int rc = set_source<R>(h, j_re, j_im);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->sc, 0, sizeof(Scalars), h->stream));
  // Algorithm init: G = P_psi 0, G_T = P* G, G* = G - G_T.
  CK(cudaMemsetAsync(h->Uw, 0, h->nvec * h->rsize, h->stream));
  sweep_source<R>(h, true, false);
  lincomb<R>(h, h->A, nullptr, nullptr, 1.0, h->Uw, 0.0, nullptr);
  sweep_free<R>(h, true);
  lincomb<R>(h, h->Rv, h->D, h->Uw, 1.0, h->A, -1.0, h->Uw);  // R = D = G*, Uw = D
  CK(cudaMemsetAsync(h->U0, 0, h->nvec * h->rsize, h->stream));
  launch_dot<R>(h->q, (const R*)h->Rv, (const R*)h->Rv, h->wdot, h->partials, h->nti, h->stream);
  launch_finalize(h->partials, nb, h->sc, 0, h->stream);
  h->launches += 2;
  rc = read_scalars<R>(h);
  if (rc) return rc;
  const double rr0 = h->sc_host->rr0;
  double rr = h->sc_host->rr;
  int it = 0;
  int status = CMCG_OK;
  bool converged = !(rr0 > 0);
  if (!std::isfinite(rr0)) status = CMCG_ERR_NONFINITE;
  while (status == CMCG_OK && !converged && it < max_iter) {
    if (std::sqrt(rr) <= tol * std::sqrt(rr0)) {
      converged = true;
      break;
    }
    // Algorithm grad on D: W_T = P D - D; A = P* W_T - W_T.
    sweep_free<R>(h, false);
    lincomb<R>(h, h->WT, h->Uw, nullptr, 1.0, h->Uw, -1.0, h->D);
    sweep_free<R>(h, true);
    launch_cg_after_adjoint<R>(h->q, (const R*)h->Uw, (const R*)h->WT, (R*)h->A, (const R*)h->D, h->wdot, h->partials,
                               h->nti, h->stream);
    launch_finalize(h->partials, nb, h->sc, 1, h->stream);
    launch_cg_update<R>(h->q, (R*)h->U0, (R*)h->Rv, (const R*)h->D, (const R*)h->A, h->wdot, h->sc, h->partials, h->nti,
                        h->stream);
    launch_finalize(h->partials, nb, h->sc, 2, h->stream);
    launch_cg_direction<R>((R*)h->D, (R*)h->Uw, (const R*)h->Rv, h->sc, h->nvec, h->stream);
    h->launches += 5;
    ++it;
    rc = read_scalars<R>(h);
    if (rc) return rc;
    if (h->sc_host->status != 0) status = h->sc_host->status;
    rr = h->sc_host->rr;
  }
  if (!converged && status == CMCG_OK && std::sqrt(rr) <= tol * std::sqrt(rr0)) converged = true;
  // Final filter F_{psi,w} U0.
  lincomb<R>(h, h->Uw, nullptr, nullptr, 1.0, h->U0, 0.0, nullptr);
  CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
  CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
  sweep_source<R>(h, true, true);
  to_ext<R>(h, (const R*)h->Fre, 6, 0, e_re, 3, 3);
  to_ext<R>(h, (const R*)h->Fim, 6, 0, e_im, 3, 3);
  to_ext<R>(h, (const R*)h->Fre, 6, 3, h_re, 3, 3);
  to_ext<R>(h, (const R*)h->Fim, 6, 3, h_im, 3, 3);
  CK(cudaEventRecord(ev1, h->stream));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (status == CMCG_OK && !converged) status = CMCG_NOT_CONVERGED;
  if (info) {
    info->iters = it;
    info->periods = 3 + 2 * it;
    info->steps_per_period = h->M;
    info->status = status;
    info->rel_residual = rr0 > 0 ? std::sqrt(std::max(rr, 0.0) / rr0) : 0.0;
    info->dt = h->dt;
    info->solve_ms = ms;
  }
  return status;
}

void free_all(cmcg_handle* h) {
  void* ptrs[] = {h->gvol, h->gface, h->nbr, h->wdot, h->e_of_i, h->inv_eps, h->Uw, h->vA, h->vB, h->ACC,
                  h->Fre, h->Fim, h->Jre, h->Jim, h->U0, h->Rv, h->D, h->A, h->WT, h->partials,
                  h->sc, h->ext0, h->ext1, h->ext2, h->ext3};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  for (auto& e : h->prof_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
}

template <typename R>
std::vector<R> cast(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

}  // namespace

extern "C" {

void cmcg_default_options(cmcg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->order = 1;
  opt->precision = CMCG_FP64;
  opt->flux = CMCG_FLUX_UPWIND;
  opt->steps_per_period = 0;
  opt->c_q = 0.0;
  opt->hbm_budget_bytes = 0;
  opt->device = 0;
}

const char* cmcg_status_string(int s) {
  switch (s) {
    case CMCG_OK: return "ok";
    case CMCG_NOT_CONVERGED: return "not converged (max_iter reached; last iterate returned)";
    case CMCG_ERR_INVALID_ARG: return "invalid argument";
    case CMCG_ERR_NONCONFORMING_MESH: return "non-conforming mesh";
    case CMCG_ERR_OUT_OF_MEMORY: return "out of device memory or over the HBM budget";
    case CMCG_ERR_UNSTABLE: return "unstable time step (energy growth)";
    case CMCG_ERR_CG_BREAKDOWN: return "conjugate-gradient breakdown ((D, A) <= 0)";
    case CMCG_ERR_NONFINITE: return "non-finite value";
    case CMCG_ERR_DEVICE_TIMEOUT: return "device wait timed out";
    case CMCG_ERR_CUDA: return "CUDA error";
    case CMCG_ERR_NO_DEVICE: return "no usable CUDA device";
    default: return "unknown status";
  }
}

int cmcg_validate(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega, const cmcg_options* opt,
                  int* steps) {
  HostLayout L;
  std::string why;
  int rc;
  try {
    rc = validate_and_layout(mesh, eps, mu, omega, opt, &L, false, &why);
  } catch (const std::bad_alloc&) {
    return CMCG_ERR_OUT_OF_MEMORY;
  } catch (...) {
    return CMCG_ERR_INVALID_ARG;
  }
  if (rc == CMCG_OK && steps) *steps = L.steps;
  return rc;
}

int cmcg_reference_matrices(int order, double* mass, double* dr, double* ds, double* dt, double* lift) {
  if (order < 1 || order > 3) return CMCG_ERR_INVALID_ARG;
  const RefMats& rm = ref_mats(order);
  const int np = rm.np, nfp = rm.nfp;
  if (mass) std::memcpy(mass, rm.M.data(), sizeof(double) * np * np);
  if (dr) std::memcpy(dr, rm.Dr.data(), sizeof(double) * np * np);
  if (ds) std::memcpy(ds, rm.Ds.data(), sizeof(double) * np * np);
  if (dt) std::memcpy(dt, rm.Dt.data(), sizeof(double) * np * np);
  if (lift) {
    // reorder each face's columns to increasing volume-node order
    for (int f = 0; f < 4; ++f) {
      std::vector<int> idx(nfp);
      for (int j = 0; j < nfp; ++j) idx[j] = j;
      std::sort(idx.begin(), idx.end(), [&](int a, int b) { return rm.fmask[f * nfp + a] < rm.fmask[f * nfp + b]; });
      for (int i = 0; i < np; ++i)
        for (int j = 0; j < nfp; ++j) lift[i * 4 * nfp + f * nfp + j] = rm.LIFT[i * 4 * nfp + f * nfp + idx[j]];
    }
  }
  return CMCG_OK;
}

int cmcg_create(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega, const cmcg_options* opt_in,
                cmcg_handle** out) {
  if (!out) return CMCG_ERR_INVALID_ARG;
  *out = nullptr;
  cmcg_options opt;
  if (opt_in) opt = *opt_in;
  else cmcg_default_options(&opt);
  cmcg_handle* h = new (std::nothrow) cmcg_handle();
  if (!h) return CMCG_ERR_OUT_OF_MEMORY;
  std::string why;
  int rc;
  try {
    rc = validate_and_layout(mesh, eps, mu, omega, &opt, &h->L, true, &why);
  } catch (const std::bad_alloc&) {
    rc = CMCG_ERR_OUT_OF_MEMORY;
  } catch (...) {
    rc = CMCG_ERR_INVALID_ARG;
  }
  if (rc) {
    delete h;
    return rc;
  }
  const HostLayout& L = h->L;
  h->device = opt.device;
  h->q = opt.order;
  h->np = np_of(opt.order);
  h->prec = opt.precision;
  h->integrator = opt.order == 1 ? 2 : 4;
  h->omega = omega;
  h->T = L.T;
  h->dt = L.dt;
  h->M = L.steps;
  h->nt = L.nt;
  h->nti = L.nti;
  h->nvec = L.nti * 6 * h->np;
  h->njvec = L.nti * 3 * h->np;
  h->rsize = opt.precision == CMCG_FP32 ? 4 : 8;
  filter_weights(h);

  const size_t extlen = size_t(L.nt) * 6 * h->np * sizeof(double);
  const size_t need = 11 * h->nvec * h->rsize + 2 * h->njvec * h->rsize + L.gvol.size() * h->rsize +
                      L.gface.size() * h->rsize + L.nbr.size() * 4 + L.wdot.size() * 8 + L.ext_of_int.size() * 4 +
                      L.nt * 8 + 4 * extlen + 4096 * 8 + sizeof(Scalars);
  h->bytes = need;
  if (opt.hbm_budget_bytes > 0 && (int64_t)need > opt.hbm_budget_bytes) {
    delete h;
    return CMCG_ERR_OUT_OF_MEMORY;
  }
  int ndev = 0;
  cudaError_t ce = cudaGetDeviceCount(&ndev);
  if (ce != cudaSuccess || ndev == 0) {
    delete h;
    return CMCG_ERR_NO_DEVICE;
  }
  if (opt.device < 0 || opt.device >= ndev) {
    delete h;
    return CMCG_ERR_INVALID_ARG;
  }
  auto fail = [&](int code) {
    free_all(h);
    delete h;
    return code;
  };
  if (cudaSetDevice(opt.device) != cudaSuccess) return fail(CMCG_ERR_CUDA);
  if ((rc = ensure_constants(opt.device, opt.order))) return fail(rc);

  auto alloc = [&](void** p, size_t bytes) -> bool { return cudaMalloc(p, bytes) == cudaSuccess; };
  const size_t vb = h->nvec * h->rsize, jb = h->njvec * h->rsize;
  bool ok = alloc(&h->gvol, L.gvol.size() * h->rsize) && alloc(&h->gface, L.gface.size() * h->rsize) &&
            alloc((void**)&h->nbr, L.nbr.size() * 4) && alloc((void**)&h->wdot, L.wdot.size() * 8) &&
            alloc((void**)&h->e_of_i, L.ext_of_int.size() * 4) && alloc((void**)&h->inv_eps, L.nt * 8) &&
            alloc(&h->Uw, vb) && alloc(&h->vA, vb) && alloc(&h->vB, vb) && alloc(&h->ACC, vb) && alloc(&h->Fre, vb) &&
            alloc(&h->Fim, vb) && alloc(&h->Jre, jb) && alloc(&h->Jim, jb) && alloc(&h->U0, vb) && alloc(&h->Rv, vb) &&
            alloc(&h->D, vb) && alloc(&h->A, vb) && alloc(&h->WT, vb) &&
            alloc((void**)&h->partials, sizeof(double) * 4096) && alloc((void**)&h->sc, sizeof(Scalars)) &&
            alloc((void**)&h->ext0, extlen) && alloc((void**)&h->ext1, extlen) && alloc((void**)&h->ext2, extlen) &&
            alloc((void**)&h->ext3, extlen);
  if (!ok) return fail(CMCG_ERR_OUT_OF_MEMORY);
  if (cudaMallocHost((void**)&h->sc_host, sizeof(Scalars)) != cudaSuccess) return fail(CMCG_ERR_OUT_OF_MEMORY);
  std::vector<double> inv_eps(L.nt);
  for (int64_t k = 0; k < L.nt; ++k) inv_eps[k] = 1.0 / eps[k];
  cudaError_t e = cudaSuccess;
  if (h->prec == CMCG_FP32) {
    auto gv = cast<float>(L.gvol), gf = cast<float>(L.gface);
    e = cudaMemcpy(h->gvol, gv.data(), gv.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->gface, gf.data(), gf.size() * 4, cudaMemcpyHostToDevice);
  } else {
    e = cudaMemcpy(h->gvol, L.gvol.data(), L.gvol.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(h->gface, L.gface.data(), L.gface.size() * 8, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemcpy(h->nbr, L.nbr.data(), L.nbr.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->wdot, L.wdot.data(), L.wdot.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->e_of_i, L.ext_of_int.data(), L.ext_of_int.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->inv_eps, inv_eps.data(), L.nt * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->ACC, 0, vb);
  if (e != cudaSuccess) return fail(cuda_fail(e));
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, opt.device) != cudaSuccess) return fail(CMCG_ERR_CUDA);
    h->nsm = nsm;
  }
  for (double& x : h->tune_us) x = -1;
  if (opt.stage_variant > 0) {
    const int nv = h->prec == CMCG_FP32 ? STAGE_VARIANTS_F32 : 1;
    const int k = opt.stage_variant - 1;
    if (k < nv) {
      h->variant = k;
    } else if (k == 3 && h->prec == CMCG_FP32) {
      h->packed_minb = 2;
    } else {
      return fail(CMCG_ERR_INVALID_ARG);
    }
  } else {
    rc = h->prec == CMCG_FP32 ? autotune<float>(h, STAGE_VARIANTS_F32) : autotune<double>(h, 1);
    if (rc) return fail(rc);
  }
  h->launches = 0;
  *out = h;
  return CMCG_OK;
}

void cmcg_destroy(cmcg_handle* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  free_all(h);
  delete h;
}

int cmcg_set_stream(cmcg_handle* h, void* stream) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  h->stream = (cudaStream_t)stream;
  return CMCG_OK;
}

int cmcg_get_sizes(const cmcg_handle* h, int64_t* nt, int* np, int* steps, double* dt, int64_t* field_len) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  if (nt) *nt = h->nt;
  if (np) *np = h->np;
  if (steps) *steps = h->M;
  if (dt) *dt = h->dt;
  if (field_len) *field_len = h->nt * 6 * h->np;
  return CMCG_OK;
}

int64_t cmcg_kernel_launches(const cmcg_handle* h) { return h ? h->launches : 0; }

int cmcg_get_tuning(const cmcg_handle* h, int* variant, double* us_per_stage) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  if (variant) *variant = h->packed_minb > 0 ? 3 : h->variant;
  if (us_per_stage)
    for (int i = 0; i < 8; ++i) us_per_stage[i] = h->tune_us[i];
  return CMCG_OK;
}

int cmcg_profile_enable(cmcg_handle* h, int on) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  prof_collect(h);
  h->prof = on != 0;
  h->prof_ms[0] = h->prof_ms[1] = 0;
  h->prof_stages[0] = h->prof_stages[1] = 0;
  return CMCG_OK;
}

int cmcg_profile_read(cmcg_handle* h, double* free_ms, int64_t* free_stages, double* source_ms,
                      int64_t* source_stages) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  prof_collect(h);
  if (free_ms) *free_ms = h->prof_ms[0];
  if (free_stages) *free_stages = h->prof_stages[0];
  if (source_ms) *source_ms = h->prof_ms[1];
  if (source_stages) *source_stages = h->prof_stages[1];
  return CMCG_OK;
}

#define DISPATCH(h, call_f, call_d) ((h)->prec == CMCG_FP32 ? (call_f) : (call_d))

int dgtd_apply(cmcg_handle* h, double t, const double* u, const double* j_re, const double* j_im, int adjoint,
               double* out) {
  if (!h || !u || !out) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(h->nt) * 6 * h->np, nj = size_t(h->nt) * 3 * h->np;
  CK(cudaMemcpyAsync(h->ext0, u, n * 8, cudaMemcpyHostToDevice, h->stream));
  if (j_re) CK(cudaMemcpyAsync(h->ext2, j_re, nj * 8, cudaMemcpyHostToDevice, h->stream));
  if (j_re && j_im) CK(cudaMemcpyAsync(h->ext3, j_im, nj * 8, cudaMemcpyHostToDevice, h->stream));
  const double* jr = j_re ? h->ext2 : nullptr;
  const double* ji = (j_re && j_im) ? h->ext3 : nullptr;
  int rc = DISPATCH(h, apply_dev<float>(h, t, h->ext0, jr, ji, adjoint, h->ext1),
                    apply_dev<double>(h, t, h->ext0, jr, ji, adjoint, h->ext1));
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, h->ext1, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

int dgtd_period_forward_device(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT,
                               double* filt_re, double* filt_im) {
  if (!h || !u0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, forward_dev<float>(h, u0, j_re, j_im, uT, filt_re, filt_im),
                  forward_dev<double>(h, u0, j_re, j_im, uT, filt_re, filt_im));
}

int dgtd_period_adjoint_device(cmcg_handle* h, const double* wT, double* w0) {
  if (!h || !wT || !w0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, adjoint_dev<float>(h, wT, w0), adjoint_dev<double>(h, wT, w0));
}

int dgtd_period_forward(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT,
                        double* filt_re, double* filt_im) {
  if (!h || !u0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(h->nt) * 6 * h->np, nj = size_t(h->nt) * 3 * h->np;
  // ext0: u0 / uT, ext1: filter re, ext2: filter im, ext3: j (re then im share ext3 halves)
  CK(cudaMemcpyAsync(h->ext0, u0, n * 8, cudaMemcpyHostToDevice, h->stream));
  const double* jr = nullptr;
  const double* ji = nullptr;
  if (j_re) {
    CK(cudaMemcpyAsync(h->ext3, j_re, nj * 8, cudaMemcpyHostToDevice, h->stream));
    jr = h->ext3;
    if (j_im) {
      CK(cudaMemcpyAsync(h->ext3 + nj, j_im, nj * 8, cudaMemcpyHostToDevice, h->stream));
      ji = h->ext3 + nj;
    }
  }
  const bool filter = filt_re && filt_im;
  int rc = DISPATCH(h, forward_dev<float>(h, h->ext0, jr, ji, h->ext0, filter ? h->ext1 : nullptr, filter ? h->ext2 : nullptr),
                    forward_dev<double>(h, h->ext0, jr, ji, h->ext0, filter ? h->ext1 : nullptr, filter ? h->ext2 : nullptr));
  if (rc) return rc;
  if (uT) CK(cudaMemcpyAsync(uT, h->ext0, n * 8, cudaMemcpyDeviceToHost, h->stream));
  if (filter) {
    CK(cudaMemcpyAsync(filt_re, h->ext1, n * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(filt_im, h->ext2, n * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

int dgtd_period_adjoint(cmcg_handle* h, const double* wT, double* w0) {
  if (!h || !wT || !w0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(h->nt) * 6 * h->np;
  CK(cudaMemcpyAsync(h->ext0, wT, n * 8, cudaMemcpyHostToDevice, h->stream));
  int rc = DISPATCH(h, adjoint_dev<float>(h, h->ext0, h->ext0), adjoint_dev<double>(h, h->ext0, h->ext0));
  if (rc) return rc;
  CK(cudaMemcpyAsync(w0, h->ext0, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

int cmcg_inner(cmcg_handle* h, const double* u, const double* v, double* out) {
  if (!h || !u || !v || !out) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(h->nt) * 6 * h->np;
  CK(cudaMemcpyAsync(h->ext0, u, n * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->ext1, v, n * 8, cudaMemcpyHostToDevice, h->stream));
  return DISPATCH(h, inner_dev<float>(h, h->ext0, h->ext1, out), inner_dev<double>(h, h->ext0, h->ext1, out));
}

int cmcg_solve_device(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
                      double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  if (!h || !j_re || !e_re || !e_im || !h_re || !h_im || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, solve_dev<float>(h, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info),
                  solve_dev<double>(h, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info));
}

int cmcg_solve(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
               double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  if (!h || !j_re || !e_re || !e_im || !h_re || !h_im || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t nj = size_t(h->nt) * 3 * h->np;
  // ext3 holds j (re, im); results go to ext0 (e_re, e_im halves) and ext1 (h_re, h_im halves)
  CK(cudaMemcpyAsync(h->ext3, j_re, nj * 8, cudaMemcpyHostToDevice, h->stream));
  const double* ji = nullptr;
  if (j_im) {
    CK(cudaMemcpyAsync(h->ext3 + nj, j_im, nj * 8, cudaMemcpyHostToDevice, h->stream));
    ji = h->ext3 + nj;
  }
  int rc = DISPATCH(h, solve_dev<float>(h, h->ext3, ji, tol, max_iter, h->ext0, h->ext0 + nj, h->ext1, h->ext1 + nj, info),
                    solve_dev<double>(h, h->ext3, ji, tol, max_iter, h->ext0, h->ext0 + nj, h->ext1, h->ext1 + nj, info));
  if (rc < 0) return rc;
  CK(cudaMemcpyAsync(e_re, h->ext0, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(e_im, h->ext0 + nj, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h_re, h->ext1, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h_im, h->ext1 + nj, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

}  // extern "C"
