// C ABI of libcmcg: handle life cycle, period sweeps and the CMCG driver.
//
// A handle holds a batch of one or more problems of the same polynomial order
// and precision (meshes, materials, frequencies and step counts may differ).
// Problems are concatenated tile-wise in the device layout; every stage launch
// covers all of them in lockstep, each problem reading its own coefficients
// (step size, source phase, filter weights, whether it is still stepping) from
// a per-launch table built once at creation.  Sweeps therefore never depend on
// host data at run time.
//
// Sweeps (Section 4.1.2, Algorithms rk2 / rk4).  The state being propagated
// lives in the work vector Uw.
//   * source-free sweeps (P_w, P*_w) use the nested form of the RK polynomial,
//     v <- U + (dt / k) B v for k = s, ..., 1, which is the same polynomial
//     sum_k (dt B)^k / k! as Algorithms rk2 / rk4 for a linear autonomous system
//     and differs from them only by rounding;
//   * sweeps with the source (P_{psi,w}, F_{psi,w}) use the same nested form with
//     a source term g_k added at nested stage k: for U' = B U + f(t), Algorithm
//     rk4 gives U_{m+1} = sum_k (dt B)^k / k! U_m + dt/6 [(f1 + 4 f2 + f4)
//     + dt B (f1 + 2 f2) + dt^2/2 B^2 (f1 + f2) + dt^3/4 B^3 f1] with f1, f2, f4
//     the source at t_m, t_m + dt/2, t_m + dt, and v_4 = U + dt/4 (B U + g_4),
//     v_k = U + dt/k (B v_{k+1} + g_k) reproduces it exactly with g_4 = f1,
//     g_3 = (f1 + f2)/2, g_2 = (f1 + 2 f2)/3, g_1 = (f1 + 4 f2 + f4)/6 (Algorithm
//     rk2 is already nested: g_2 = f1, g_1 = f2).  No accumulator vector is
//     kept.  The first nested stage evaluates Phi(t_m, U_m) itself, so the
//     filter is accumulated on the fly there and once more at t_M
//     (Eq. filtering_RK2 / filtering_RK4, each with the 2/T of Eq. filter).
// CMCG (Section 2.2, Algorithms init / grad / cmcg) runs in residual form from
// U0 = 0 for every problem: G = P_psi 0, G* = G - P* G, R = D = G*, then per
// iteration W_T = P D - D, A = P* W_T - W_T, alpha = |R|^2 / (D, A),
// U0 += alpha D, R -= alpha A, beta = |R_new|^2 / |R|^2, D = R + beta D.  The
// scalars are FP64 and stay on the device, one set per problem; a problem
// whose residual meets the tolerance stops sweeping and updating.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include <nvtx3/nvToolsExt.h>

#include "common.h"

using namespace cmcg;

namespace {
// NVTX range for the lifetime of a scope (host side: sweeps, solve phases, slot rounds); free
// when no profiling tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
}  // namespace

namespace {

// An impedance face of a problem: what its boundary data need on the host.
struct ImpFace {
  int64_t it = 0;        // internal tetrahedron (handle-wide index)
  int32_t ext = 0;       // external tetrahedron within its problem
  int f = 0;             // face
  double n[3] = {0, 0, 0};
  double aE = 0, bH = 0;  // flux coefficients of the E rows (tangential jump) and H rows (n x jump)
};

struct Prob {
  int64_t nt = 0;                     // external tetrahedra
  int64_t tet0 = 0, nti = 0;          // internal range
  int64_t tile0 = 0, ntiles = 0;
  int64_t ext0 = 0;                   // prefix of external tetrahedra
  int M = 0;
  double dt = 0, T = 0, omega = 0;
  std::vector<std::complex<double>> fa, fb;  // filter weights per step 0..M (with 2/T)
  std::vector<ImpFace> imp;                   // impedance faces
  bool has_bdata = false;                     // boundary data set (cmcg_set_boundary_data)
  bool has_sigma = false;                     // conductivity set (cmcg_set_conductivity)
  std::vector<int32_t> ext_of_int;            // internal (problem-local) -> external tetrahedron (-1 padding)
  std::vector<int32_t> int_of_ext;            // external -> internal (problem-local)
};

}  // namespace

struct cmcg_handle {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  int q = 1, np = 4, prec = CMCG_FP64, s = 2, nprob = 1;
  std::vector<Prob> P;
  int64_t nti = 0, ntiles = 0, nvec = 0, njvec = 0, nt_total = 0;
  size_t rsize = 8;
  int maxM = 0;
  // device geometry
  void *gvol = nullptr, *gface = nullptr;
  int32_t* nbr = nullptr;
  double* wdot = nullptr;
  int32_t* e_of_i = nullptr;  // internal tet -> external index within its problem (-1 = padding)
  int32_t* tprob = nullptr;   // problem of each tile (nullptr when nprob == 1)
  double* inv_eps = nullptr;  // external order, problems concatenated
  // vectors
  void *Uw = nullptr, *vA = nullptr, *vB = nullptr, *Fre = nullptr, *Fim = nullptr;
  void *Jre = nullptr, *Jim = nullptr;
  void *Bre = nullptr, *Bim = nullptr;  // lifted impedance-face data, all 6 rows (allocated on first use)
  void *U0 = nullptr, *Rv = nullptr, *D = nullptr, *A = nullptr, *WT = nullptr;
  // CG
  double* partials = nullptr;
  Scalars* sc = nullptr;
  Scalars* sc_host = nullptr;  // pinned
  int32_t* pactive = nullptr;
  int32_t* pactive_host = nullptr;  // pinned
  int32_t* used = nullptr;          // problems taking part in the current solve
  int32_t* used_host = nullptr;     // pinned
  int64_t* bt_tet0 = nullptr;
  int32_t *bt_ntet = nullptr, *bt_prob = nullptr, *bt_pb0 = nullptr;
  BlockTable bt{};
  // per-launch coefficient tables
  void *tab_free = nullptr, *tab_src = nullptr, *tab_srcf = nullptr, *tab_one = nullptr;
  int L_free = 0, L_src = 0, L_srcf = 0;
  // staging for host I/O (nt_total * 6 * np doubles each)
  double *ext0 = nullptr, *ext1 = nullptr, *ext2 = nullptr, *ext3 = nullptr;
  int64_t launches = 0;
  size_t bytes = 0;
  bool has_bdata = false;  // some problem has boundary data
  bool has_sigma = false;  // some problem has a conductivity
  // Sharded handle (cmcg_create_sharded): the problems are the parts of one mesh, each with its
  // ghost layer; ghosts receive their owners' values after every stage and the CG reductions
  // sum over all parts.
  bool coupled = false;
  int64_t nt_global = 0;
  int64_t nhalo = 0;
  int64_t *halo_dst = nullptr, *halo_src = nullptr;  // internal tetrahedra: ghost <- owner
  int32_t *g_in = nullptr, *g_out = nullptr;          // internal -> global tetrahedron (g_out: owned only)
  double* inv_eps_g = nullptr;                        // 1 / eps by global tetrahedron
  // Several harmonics in one solve (cmcg_solve_multifreq): while mf_nharm > 0 the source sweeps
  // read mf_nharm sources from Jm_re / Jm_im (njvec values apart) with the per-launch harmonic
  // coefficients mf_hcs, and filtered sweeps use the filter table mf_tab of the harmonic being read.
  int mf_nharm = 0, mf_cap = 0;
  void *Jm_re = nullptr, *Jm_im = nullptr, *mf_hcs = nullptr, *mf_tab = nullptr;
  double* mf_src = nullptr;  // host sources of cmcg_solve_multifreq, on the device
  size_t mf_src_len = 0;
  // Slots (continuous batching, cmcg_slot_*): phase of every problem and the per-phase masks.
  std::vector<int> slot_phase;
  std::vector<cmcg_info> slot_info;
  int32_t* slot_masks = nullptr;       // device [3][nprob]: admitted, adjoint sweep, filter pending
  int32_t* slot_masks_host = nullptr;  // pinned
  // CUDA graphs of whole sweeps, captured on first use on a private stream and launched on
  // `stream`; key: sweep kind, mask pointer, boundary data present.
  bool graphs = true;
  cudaStream_t cap_stream = nullptr;
  std::map<std::tuple<int, const void*, bool>, cudaGraphExec_t> graph_exec;
  int form = 0;      // stage-kernel form (see launch_stage)
  bool pdl = false;  // stages launched with programmatic stream serialisation
  double tune_us[10];     // [0..6] per form, [7] the chosen form with overlapped launches, [8..9] unused
  int32_t* err = nullptr;       // device status word of the stage kernels' bounded waits
  int32_t* err_host = nullptr;  // pinned
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

#define CK(expr)                                 \
  do {                                           \
    cudaError_t e_ = (expr);                     \
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
void filter_weights(Prob& P, int integrator) {
  const int M = P.M;
  const double dt = P.dt, w = P.omega, c = 2.0 / P.T;
  P.fa.assign(M + 1, 0.0);
  P.fb.assign(M + 1, 0.0);
  using cd = std::complex<double>;
  if (integrator == 2) {
    for (int m = 0; m <= M; ++m) {
      const double wt = (m == 0 || m == M) ? 0.5 : 1.0;
      P.fa[m] = c * dt * wt * std::exp(cd(0, -w * m * dt));
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
    P.fa[m - 1] += c * e * x00;
    P.fa[m] += c * e * x01;
    P.fb[m - 1] += c * e * x10;
    P.fb[m] += c * e * x11;
  }
}

// Coefficient tables.  Launch l of a sweep is nested stage r = l % s of step m = l / s:
// out = U + dt / (s - r) Phi.  In source sweeps Phi carries the source combination g of
// nested stage s - r (see the top of this file): Re(J e^{i w t}) summed with the weights
// below over the times t_m + {0, dt/2, dt} (the stage times of Algorithms rk2 / rk4).
constexpr double SRC_OFF[3] = {0.0, 0.5, 1.0};
constexpr double SRC_W4[4][3] = {{1.0, 0.0, 0.0}, {0.5, 0.5, 0.0}, {1.0 / 3.0, 2.0 / 3.0, 0.0},
                                 {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0}};
constexpr double SRC_W2[2][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0, 0.0}};

// The source phase of launch r: sum_j W[r][j] (cos, sin)(w (t_m + SRC_OFF[j] dt)).
void source_phase(int s, int r, double dt, double t_m, double w, double* cs, double* sn) {
  const double* W = s == 4 ? SRC_W4[r] : SRC_W2[r];
  *cs = 0.0;
  *sn = 0.0;
  for (int j = 0; j < 3; ++j) {
    if (W[j] == 0.0) continue;
    const double t = t_m + SRC_OFF[j] * dt;
    *cs += W[j] * std::cos(w * t);
    *sn += W[j] * std::sin(w * t);
  }
}

template <typename R>
void source_coef(int s, int r, double dt, double t_m, double w, StageCoef<R>& c) {
  double cs, sn;
  source_phase(s, r, dt, t_m, w, &cs, &sn);
  c.c_out = R(dt / (s - r));
  c.s_cos = R(cs);
  c.s_sin = R(sn);
}

template <typename R>
int build_tables(cmcg_handle* h) {
  const int s = h->s, np_ = h->nprob;
  h->L_free = h->maxM * s;
  h->L_src = h->maxM * s;
  h->L_srcf = h->maxM * s + 1;
  std::vector<StageCoef<R>> tf(size_t(h->L_free) * np_), ts(size_t(h->L_src) * np_), tsf(size_t(h->L_srcf) * np_);
  StageCoef<R> zero;
  std::memset(&zero, 0, sizeof(zero));
  for (int l = 0; l < h->L_srcf; ++l) {
    const int m = l / s, r = l % s;
    for (int p = 0; p < np_; ++p) {
      const Prob& P = h->P[p];
      if (l < h->L_free) {
        StageCoef<R> c = zero;
        if (m < P.M) {
          c.active = 1;
          c.c_out = R(P.dt / (s - r));
        }
        tf[size_t(l) * np_ + p] = c;
        StageCoef<R> cs = zero;
        if (m < P.M) {
          cs.active = 1;
          source_coef<R>(s, r, P.dt, m * P.dt, P.omega, cs);
        }
        ts[size_t(l) * np_ + p] = cs;
      }
      StageCoef<R> cf = zero;
      if (m < P.M || (m == P.M && r == 0)) {  // the extra launch at t_M evaluates Phi_M for the filter
        cf.active = 1;
        source_coef<R>(s, r, P.dt, m * P.dt, P.omega, cf);
        if (r == 0) {
          cf.fa_re = R(P.fa[m].real());
          cf.fa_im = R(P.fa[m].imag());
          cf.fb_re = R(P.fb[m].real());
          cf.fb_im = R(P.fb[m].imag());
        }
      }
      tsf[size_t(l) * np_ + p] = cf;
    }
  }
  const size_t sz = sizeof(StageCoef<R>);
  CK(cudaMalloc(&h->tab_free, tf.size() * sz));
  CK(cudaMalloc(&h->tab_src, ts.size() * sz));
  CK(cudaMalloc(&h->tab_srcf, tsf.size() * sz));
  CK(cudaMalloc(&h->tab_one, size_t(np_) * sz));
  CK(cudaMemcpy(h->tab_free, tf.data(), tf.size() * sz, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->tab_src, ts.data(), ts.size() * sz, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->tab_srcf, tsf.data(), tsf.size() * sz, cudaMemcpyHostToDevice));
  h->bytes += (tf.size() + ts.size() + tsf.size() + np_) * sz;
  return CMCG_OK;
}

template <typename R>
const StageCoef<R>* tab(void* t, int l, int nprob) {
  return static_cast<const StageCoef<R>*>(t) + size_t(l) * nprob;
}

template <typename R>
void stage(cmcg_handle* h, StageArgs<R>& a, cudaStream_t st) {
  a.gvol = (const R*)h->gvol;
  a.gface = (const R*)h->gface;
  a.nbr = h->nbr;
  a.nti = h->nti;
  a.err = h->err;
  a.sigma = h->has_sigma ? 1 : 0;
  a.tprob = h->tprob;
  if (h->q == 1) launch_stage<1, R>(a, st, h->form, h->pdl);
  else if (h->q == 2) launch_stage<2, R>(a, st, h->form, h->pdl);
  else launch_stage<3, R>(a, st, h->form, h->pdl);
}
template <typename R>
void stage(cmcg_handle* h, StageArgs<R>& a) {
  stage<R>(h, a, h->stream);
  h->launches++;
}

// Sharded handles: every ghost takes its owner's values of the field a stage has just written.
template <typename R>
void halo(cmcg_handle* h, R* v, cudaStream_t st) {
  if (!h->coupled || !v || h->nhalo == 0) return;
  launch_halo<R>(v, h->halo_dst, h->halo_src, h->nhalo, h->np, st);
}

// Runs `emit(stream)` (a fixed sequence of `n` stage launches) on the handle's stream, from a
// CUDA graph captured at its first use under `key`; if capture or instantiation is refused,
// the handle stops using graphs and launches directly.
template <typename F>
void run_sweep(cmcg_handle* h, std::tuple<int, const void*, bool> key, int n, F&& emit) {
  if (h->graphs) {
    auto it = h->graph_exec.find(key);
    if (it == h->graph_exec.end()) {
      cudaGraphExec_t exec = nullptr;
      bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        emit(h->cap_stream);
        cudaGraph_t g = nullptr;
        ok = cudaStreamEndCapture(h->cap_stream, &g) == cudaSuccess && g;
        if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      if (!ok) {
        cudaGetLastError();  // clear the refusal; fall back to direct launches
        h->graphs = false;
      } else {
        it = h->graph_exec.emplace(key, exec).first;
      }
    }
    if (h->graphs) {
      cudaGraphLaunch(it->second, h->stream);
      h->launches += n;
      return;
    }
  }
  emit(h->stream);
  h->launches += n;
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

// Source-free sweep of Uw in place (nested RK form); adjoint flips the magnetic
// sign.  pactive: skip problems whose CG has stopped (nullptr: sweep all).
template <typename R>
void sweep_free(cmcg_handle* h, bool adjoint, const int32_t* pactive) {
  Range rg(adjoint ? "cmcg: adjoint sweep" : "cmcg: forward sweep");
  cmcg_handle::SweepEv* pe = prof_begin(h, false);
  R* Uw = (R*)h->Uw;
  R* vA = (R*)h->vA;
  R* vB = (R*)h->vB;
  const int s = h->s;
  run_sweep(h, std::make_tuple(adjoint ? 1 : 0, (const void*)pactive, false), h->L_free, [&](cudaStream_t st) {
    for (int l = 0; l < h->L_free; ++l) {
      const int r = l % s;
      StageArgs<R> a = blank<R>();
      a.vin = r == 0 ? Uw : (r % 2 == 1 ? vA : vB);
      a.base = Uw;
      a.out = r == s - 1 ? Uw : (r % 2 == 0 ? vA : vB);
      a.sH = adjoint ? R(-1) : R(1);
      a.coef = tab<R>(h->tab_free, l, h->nprob);
      a.pactive = pactive;
      stage<R>(h, a, st);
      halo<R>(h, a.out, st);
    }
  });
  prof_end(h, pe);
}

// Sweep with source (Algorithms rk2 / rk4 in the nested form with the source combinations
// of source_coef) of Uw in place; optional on-the-fly filter at the first nested stage of
// every step (one extra launch evaluates Phi at t_M).
template <typename R>
void sweep_source(cmcg_handle* h, bool with_source, bool filter, const int32_t* mask = nullptr) {
  Range rg(filter ? "cmcg: filtered source sweep" : "cmcg: source sweep");
  cmcg_handle::SweepEv* pe = prof_begin(h, true);
  R* Uw = (R*)h->Uw;
  R* vA = (R*)h->vA;
  R* vB = (R*)h->vB;
  const int s = h->s;
  const int L = filter ? h->L_srcf : h->L_src;
  const int K = with_source ? h->mf_nharm : 0;
  void* table = filter ? (K > 0 ? h->mf_tab : h->tab_srcf) : h->tab_src;
  const int kind = 2 + (filter ? 1 : 0) + (with_source ? 0 : 2);
  auto emit = [&](cudaStream_t st) {
  for (int l = 0; l < L; ++l) {
    const int r = l % s;
    StageArgs<R> a = blank<R>();
    a.vin = r == 0 ? Uw : (r % 2 == 1 ? vA : vB);  // the buffers of sweep_free
    a.base = Uw;
    a.out = r == s - 1 ? Uw : (r % 2 == 0 ? vA : vB);
    if (with_source) {
      a.jre = (const R*)(K > 0 ? h->Jm_re : h->Jre);
      a.jim = (const R*)(K > 0 ? h->Jm_im : h->Jim);
      if (K > 0) {
        a.nharm = K;
        a.jstride = h->njvec;
        a.hcs = (const R*)h->mf_hcs + size_t(l) * 2 * K;
      }
      if (h->has_bdata) {
        a.bre = (const R*)h->Bre;
        a.bim = (const R*)h->Bim;
      }
    }
    if (filter && r == 0) {
      a.fre = (R*)h->Fre;
      a.fim = (R*)h->Fim;
    }
    a.coef = tab<R>(table, l, h->nprob);
    a.pactive = mask;
    stage<R>(h, a, st);
    halo<R>(h, a.out, st);
  }
  };
  if (K > 0) {  // several harmonics: launched directly (their tables change from call to call)
    emit(h->stream);
    h->launches += L;
  } else {
    run_sweep(h, std::make_tuple(kind, (const void*)mask, with_source && h->has_bdata), L, emit);
  }
  prof_end(h, pe);
}

// Times the stage-kernel forms on this batch with a nested source-free stage
// on zero fields (3 warm-up + 12 timed launches each) and keeps the fastest;
// tune_us[f] is the time of form f (-1: not timed or rejected by the device).
template <typename R>
int autotune(cmcg_handle* h, int nforms, int overlap) {
  for (double& x : h->tune_us) x = -1;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaMemsetAsync(h->Uw, 0, h->nvec * h->rsize, h->stream));
  CK(cudaMemsetAsync(h->vB, 0, h->nvec * h->rsize, h->stream));
  const int64_t launches0 = h->launches;
  auto time_one = [&](double* us) -> int {
    auto run = [&](int n) {
      for (int k = 0; k < n; ++k) {
        StageArgs<R> a = blank<R>();
        a.vin = (const R*)h->Uw;
        a.base = (const R*)h->vB;
        a.out = (R*)h->vA;
        a.coef = tab<R>(h->tab_free, 0, h->nprob);
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
  double best = 1e300;
  int bestf = 0;
  h->pdl = false;
  for (int f = 0; f < nforms; ++f) {
    h->form = f;
    double us;
    int rc = time_one(&us);
    if (rc) return rc;
    h->tune_us[f] = us;
    if (us >= 0 && us < best) {
      best = us;
      bestf = f;
    }
  }
  h->form = bestf;
  if (overlap == 0) {  // the chosen form with overlapped stage launches
    h->pdl = true;
    double us;
    int rc = time_one(&us);
    if (rc) return rc;
    h->tune_us[7] = us;
    h->pdl = us >= 0 && us < best;
  } else {
    h->pdl = overlap == 1;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->launches = launches0;
  CK(cudaGetLastError());
  return CMCG_OK;
}

// Per-problem layout conversion.
// (For a sharded handle the external arrays are the global mesh's: every part reads its owned
// and ghost tetrahedra and writes its owned ones.)
template <typename R>
void to_int(cmcg_handle* h, int p, const double* ext, int ncomp_ext, void* in, int ncomp_in, int cnt,
            const double* per_tet) {
  const Prob& P = h->P[p];
  R* base = (R*)in + P.tile0 * int64_t(ncomp_in) * h->np * TILE;
  const int32_t* map = h->coupled ? h->g_in + P.tet0 : h->e_of_i + P.tet0;
  const double* pt = per_tet ? (h->coupled ? h->inv_eps_g : per_tet + P.ext0) : nullptr;
  launch_to_internal<R>(ext, ncomp_ext, 0, base, ncomp_in, 0, cnt, map, P.nti, h->np, 1.0, pt, h->stream);
  h->launches++;
}
template <typename R>
void to_ext(cmcg_handle* h, int p, const void* in, int ncomp_in, int c_in0, double* ext, int ncomp_ext, int cnt) {
  const Prob& P = h->P[p];
  const R* base = (const R*)in + P.tile0 * int64_t(ncomp_in) * h->np * TILE;
  const int32_t* map = h->coupled ? h->g_out + P.tet0 : h->e_of_i + P.tet0;
  launch_to_external<R>(base, ncomp_in, c_in0, ext, ncomp_ext, 0, cnt, map, P.nti, h->np, h->stream);
  h->launches++;
}
// Number of problems a single-problem entry point converts: all parts of a sharded handle.
int nconv(const cmcg_handle* h) { return h->coupled ? h->nprob : 1; }
// Tetrahedra of the external (caller's) arrays of a single-problem entry point.
int64_t ext_nt(const cmcg_handle* h) { return h->coupled ? h->nt_global : h->nt_total; }
template <typename R>
void lincomb(cmcg_handle* h, void* o1, void* o2, void* o3, double a, const void* x, double b, const void* y) {
  launch_lincomb3<R>((R*)o1, (R*)o2, (R*)o3, a, (const R*)x, b, (const R*)y, h->nvec, h->stream);
  h->launches++;
}

template <typename R>
int set_source(cmcg_handle* h, const double* const* j_re, const double* const* j_im, int nused = -1) {
  for (int p = 0; p < (nused < 0 ? h->nprob : nused); ++p) {
    to_int<R>(h, p, j_re[p], 3, h->Jre, 3, 3, h->inv_eps);
    const double* ji = j_im ? j_im[p] : nullptr;
    if (ji) {
      to_int<R>(h, p, ji, 3, h->Jim, 3, 3, h->inv_eps);
    } else {
      const Prob& P = h->P[p];
      CK(cudaMemsetAsync((char*)h->Jim + P.tile0 * 3 * h->np * TILE * h->rsize, 0,
                         size_t(P.ntiles) * 3 * h->np * TILE * h->rsize, h->stream));
    }
  }
  return CMCG_OK;
}

// Device status after a synchronised sweep: CMCG_ERR_DEVICE_TIMEOUT if a stage kernel's bounded
// wait ran out (the word is then cleared for the next call).
int check_err(cmcg_handle* h) {
  CK(cudaMemcpyAsync(h->err_host, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*h->err_host == 0) return CMCG_OK;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_ERR_DEVICE_TIMEOUT;
}

// Device-pointer period sweeps of a one-problem handle.
template <typename R>
int forward_dev(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT, double* fre,
                double* fim) {
  for (int p = 0; p < nconv(h); ++p) to_int<R>(h, p, u0, 6, h->Uw, 6, 6, nullptr);
  const bool filter = fre && fim;
  if (j_re) {
    std::vector<const double*> jr(size_t(h->nprob), j_re), ji(size_t(h->nprob), j_im);
    int rc = set_source<R>(h, jr.data(), ji.data(), nconv(h));
    if (rc) return rc;
  }
  if (filter) {
    CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
    CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
  }
  if (j_re || filter) sweep_source<R>(h, j_re != nullptr, filter);
  else sweep_free<R>(h, false, nullptr);
  for (int p = 0; p < nconv(h); ++p) {
    if (uT) to_ext<R>(h, p, h->Uw, 6, 0, uT, 6, 6);
    if (filter) {
      to_ext<R>(h, p, h->Fre, 6, 0, fre, 6, 6);
      to_ext<R>(h, p, h->Fim, 6, 0, fim, 6, 6);
    }
  }
  CK(cudaGetLastError());
  return check_err(h);
}

template <typename R>
int adjoint_dev(cmcg_handle* h, const double* wT, double* w0) {
  for (int p = 0; p < nconv(h); ++p) to_int<R>(h, p, wT, 6, h->Uw, 6, 6, nullptr);
  sweep_free<R>(h, true, nullptr);
  for (int p = 0; p < nconv(h); ++p) to_ext<R>(h, p, h->Uw, 6, 0, w0, 6, 6);
  CK(cudaGetLastError());
  return check_err(h);
}

template <typename R>
int apply_dev(cmcg_handle* h, double t, const double* u, const double* j_re, const double* j_im, int adjoint,
              double* out) {
  for (int p = 0; p < nconv(h); ++p) to_int<R>(h, p, u, 6, h->Uw, 6, 6, nullptr);
  CK(cudaMemsetAsync(h->vB, 0, h->nvec * h->rsize, h->stream));
  StageCoef<R> c;
  std::memset(&c, 0, sizeof(c));
  c.active = 1;
  c.c_out = R(1);
  c.s_cos = R(std::cos(h->P[0].omega * t));
  c.s_sin = R(std::sin(h->P[0].omega * t));
  const std::vector<StageCoef<R>> cs(size_t(h->nprob), c);  // every part of a sharded handle
  CK(cudaMemcpy(h->tab_one, cs.data(), sizeof(c) * cs.size(), cudaMemcpyHostToDevice));
  StageArgs<R> a = blank<R>();
  a.vin = (const R*)h->Uw;
  a.base = (const R*)h->vB;
  a.out = (R*)h->vA;
  a.sH = adjoint ? R(-1) : R(1);
  a.coef = (const StageCoef<R>*)h->tab_one;
  if (j_re && !adjoint) {
    std::vector<const double*> jr(size_t(h->nprob), j_re), ji(size_t(h->nprob), j_im);
    int rc = set_source<R>(h, jr.data(), ji.data(), nconv(h));
    if (rc) return rc;
    a.jre = (const R*)h->Jre;
    a.jim = (const R*)h->Jim;
    if (h->has_bdata) {
      a.bre = (const R*)h->Bre;
      a.bim = (const R*)h->Bim;
    }
  }
  stage<R>(h, a);
  for (int p = 0; p < nconv(h); ++p) to_ext<R>(h, p, h->vA, 6, 0, out, 6, 6);
  CK(cudaGetLastError());
  return check_err(h);
}

template <typename R>
int inner_dev(cmcg_handle* h, const double* u, const double* v, double* out) {
  for (int p = 0; p < nconv(h); ++p) {
    to_int<R>(h, p, u, 6, h->Uw, 6, 6, nullptr);
    to_int<R>(h, p, v, 6, h->vA, 6, 6, nullptr);
  }
  launch_dot<R>(h->q, (const R*)h->Uw, (const R*)h->vA, h->wdot, h->partials, h->bt, h->stream);
  launch_finalize(h->partials, h->bt, h->sc, nullptr, nullptr, 3, 0.0, h->stream);
  h->launches += 2;
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->sc_host[0].rr_new;
  return CMCG_OK;
}

int read_state(cmcg_handle* h) {
  CK(cudaMemcpyAsync(h->sc_host, h->sc, sizeof(Scalars) * h->nprob, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->pactive_host, h->pactive, sizeof(int32_t) * h->nprob, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->err_host, h->err, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (*h->err_host == 0) return CMCG_OK;
  CK(cudaMemsetAsync(h->err, 0, sizeof(int32_t), h->stream));  // cleared for the next call
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_ERR_DEVICE_TIMEOUT;
}


template <typename R>
int cg_phase(cmcg_handle* h, const int32_t* mask, double tol, int max_iter);
int report(cmcg_handle* h, int nused, double tol, float ms, int extra_periods, cmcg_info* info);

// CMCG for problems [0, nused) of the handle (the others are skipped by every
// kernel); j, e, h: one device pointer per used problem.
template <typename R>
int solve_dev(cmcg_handle* h, int nused, const double* const* j_re, const double* const* j_im, double tol,
              int max_iter, double* const* e_re, double* const* e_im, double* const* h_re, double* const* h_im,
              cmcg_info* info) {
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, h->stream));
  for (int p = 0; p < h->nprob; ++p) h->used_host[p] = p < nused ? 1 : 0;
  CK(cudaMemcpyAsync(h->used, h->used_host, sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, h->stream));
  const int32_t* mask = nused < h->nprob ? h->used : nullptr;
  int rc = set_source<R>(h, j_re, j_im, nused);
  if (rc) return rc;
  if ((rc = cg_phase<R>(h, mask, tol, max_iter))) return rc;
  // Final filter F_{psi,w} U0 for every used problem.
  lincomb<R>(h, h->Uw, nullptr, nullptr, 1.0, h->U0, 0.0, nullptr);
  CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
  CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
  sweep_source<R>(h, true, true, mask);
  for (int p = 0; p < nused; ++p) {
    to_ext<R>(h, p, h->Fre, 6, 0, e_re[p], 3, 3);
    to_ext<R>(h, p, h->Fim, 6, 0, e_im[p], 3, 3);
    to_ext<R>(h, p, h->Fre, 6, 3, h_re[p], 3, 3);
    to_ext<R>(h, p, h->Fim, 6, 3, h_im[p], 3, 3);
  }
  CK(cudaEventRecord(ev1, h->stream));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  if ((rc = check_err(h))) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return report(h, nused, tol, ms, 0, info);
}

// Algorithms init and cmcg (residual form) on the sources already in place, for the problems
// of `mask` (nullptr: all); U0 holds the result.
template <typename R>
int cg_phase(cmcg_handle* h, const int32_t* mask, double tol, int max_iter) {
  Range rg("cmcg: init and CG");
  int rc = CMCG_OK;
  CK(cudaMemsetAsync(h->sc, 0, sizeof(Scalars) * h->nprob, h->stream));
  // Algorithm init: G = P_psi 0, G_T = P* G, G* = G - G_T.
  CK(cudaMemsetAsync(h->Uw, 0, h->nvec * h->rsize, h->stream));
  sweep_source<R>(h, true, false, mask);
  lincomb<R>(h, h->A, nullptr, nullptr, 1.0, h->Uw, 0.0, nullptr);
  sweep_free<R>(h, true, mask);
  lincomb<R>(h, h->Rv, h->D, h->Uw, 1.0, h->A, -1.0, h->Uw);  // R = D = G*, Uw = D
  CK(cudaMemsetAsync(h->U0, 0, h->nvec * h->rsize, h->stream));
  launch_dot<R>(h->q, (const R*)h->Rv, (const R*)h->Rv, h->wdot, h->partials, h->bt, h->stream);
  launch_finalize(h->partials, h->bt, h->sc, h->pactive, h->used, 0, tol, h->stream);
  h->launches += 2;
  rc = read_state(h);
  if (rc) return rc;
  auto any_active = [&]() {
    for (int p = 0; p < h->nprob; ++p)
      if (h->pactive_host[p]) return true;
    return false;
  };
  int it = 0;
  while (any_active() && it < max_iter) {
    Range rit("cmcg: CG iteration");
    // Algorithm grad on D: W_T = P D - D; A = P* W_T - W_T.
    sweep_free<R>(h, false, h->pactive);
    lincomb<R>(h, h->WT, h->Uw, nullptr, 1.0, h->Uw, -1.0, h->D);
    sweep_free<R>(h, true, h->pactive);
    launch_cg_after_adjoint<R>(h->q, (const R*)h->Uw, (const R*)h->WT, (R*)h->A, (const R*)h->D, h->wdot, h->partials,
                               h->bt, h->pactive, h->stream);
    launch_finalize(h->partials, h->bt, h->sc, h->pactive, nullptr, 1, tol, h->stream);
    launch_cg_update<R>(h->q, (R*)h->U0, (R*)h->Rv, (const R*)h->D, (const R*)h->A, h->wdot, h->sc, h->partials, h->bt,
                        h->pactive, h->stream);
    launch_finalize(h->partials, h->bt, h->sc, h->pactive, nullptr, 2, tol, h->stream);
    // problems that just converged keep D; the others get D = R + beta D, Uw = D
    launch_cg_direction<R>((R*)h->D, (R*)h->Uw, (const R*)h->Rv, h->sc, h->tprob, h->pactive, h->nvec, h->np,
                           h->stream);
    h->launches += 5;
    ++it;
    rc = read_state(h);
    if (rc) return rc;
  }
  return CMCG_OK;
}

// Reports of problems [0, nused) after a synchronised solve; extra_periods: filtered sweeps
// beyond the one of Algorithm cmcg.  Returns the most severe status.
int report(cmcg_handle* h, int nused, double tol, float ms, int extra_periods, cmcg_info* info) {
  int worst = CMCG_OK;
  for (int p = 0; p < nused; ++p) {
    const Scalars& S = h->sc_host[p];
    int st = S.status;
    const bool conv = S.rr0 > 0 ? std::sqrt(std::max(S.rr, 0.0)) <= tol * std::sqrt(S.rr0) : true;
    if (st == CMCG_OK && !conv) st = CMCG_NOT_CONVERGED;
    if (st < 0) {
      if (worst >= 0 || st < worst) worst = st;
    } else if (worst >= 0 && st > worst) {
      worst = st;
    }
    if (info) {
      info[p].iters = S.iters;
      info[p].periods = 3 + 2 * S.iters + extra_periods;
      info[p].steps_per_period = h->P[p].M;
      info[p].status = st;
      info[p].rel_residual = S.rr0 > 0 ? std::sqrt(std::max(S.rr, 0.0) / S.rr0) : 0.0;
      info[p].dt = h->P[p].dt;
      info[p].solve_ms = ms;
    }
  }
  return worst;
}

// Several frequencies in one solve (the one-shot remark of the Conclusion, Section 7): the
// handle's omega is the base frequency w0; harmonic k_h w0 has the source j_h.  CMCG runs once on
// the period T0 = 2 pi / w0 of the summed source; then one filtered sweep from U0 per harmonic,
// each with the filter weights of its frequency k_h w0 over T0 (Eq. filter, Section 5.4),
// returns that frequency's time-harmonic field.  Sources j_h and results are device pointers;
// `sink(h_index)` runs after harmonic h's results are written (host entry points copy them out).
template <typename R, typename Sink>
int solve_multi_dev(cmcg_handle* h, int K, const int* harm, const double* const* j_re, const double* const* j_im,
                    double tol, int max_iter, double* e_re, double* e_im, double* h_re, double* h_im, Sink&& sink,
                    cmcg_info* info) {
  Prob& P = h->P[0];
  const size_t vb = size_t(h->njvec) * h->rsize;
  if (K > h->mf_cap) {  // K sources and the per-launch harmonic coefficients (kept for later calls)
    if (h->Jm_re) cudaFree(h->Jm_re);
    if (h->Jm_im) cudaFree(h->Jm_im);
    if (h->mf_hcs) cudaFree(h->mf_hcs);
    h->Jm_re = h->Jm_im = h->mf_hcs = nullptr;
    h->mf_cap = 0;
    if (cudaMalloc(&h->Jm_re, vb * K) != cudaSuccess || cudaMalloc(&h->Jm_im, vb * K) != cudaSuccess ||
        cudaMalloc(&h->mf_hcs, size_t(h->L_srcf) * 2 * K * h->rsize) != cudaSuccess)
      return CMCG_ERR_OUT_OF_MEMORY;
    h->mf_cap = K;
    h->bytes += 2 * vb * K + size_t(h->L_srcf) * 2 * K * h->rsize;
  }
  if (!h->mf_tab) {
    if (cudaMalloc(&h->mf_tab, size_t(h->L_srcf) * sizeof(StageCoef<R>)) != cudaSuccess) return CMCG_ERR_OUT_OF_MEMORY;
    h->bytes += size_t(h->L_srcf) * sizeof(StageCoef<R>);
  }
  // source phase of every harmonic at every launch (the nested-stage combination of source_coef)
  const int s = h->s;
  std::vector<R> hcs(static_cast<size_t>(h->L_srcf) * 2 * K);
  for (int l = 0; l < h->L_srcf; ++l) {
    const int m = l / s, r = l % s;
    for (int k = 0; k < K; ++k) {
      double cs, sn;
      source_phase(s, r, P.dt, m * P.dt, harm[k] * P.omega, &cs, &sn);
      hcs[(size_t(l) * K + k) * 2] = R(cs);
      hcs[(size_t(l) * K + k) * 2 + 1] = R(sn);
    }
  }
  CK(cudaMemcpyAsync(h->mf_hcs, hcs.data(), hcs.size() * sizeof(R), cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t ev0, ev1;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, h->stream));
  for (int k = 0; k < K; ++k) {
    void* jr = static_cast<char*>(h->Jm_re) + vb * k;
    void* ji = static_cast<char*>(h->Jm_im) + vb * k;
    to_int<R>(h, 0, j_re[k], 3, jr, 3, 3, h->inv_eps);
    if (j_im && j_im[k]) to_int<R>(h, 0, j_im[k], 3, ji, 3, 3, h->inv_eps);
    else CK(cudaMemsetAsync(ji, 0, vb, h->stream));
  }
  h->used_host[0] = 1;  // the problem takes part (read by the first reduction of the CG phase)
  CK(cudaMemcpyAsync(h->used, h->used_host, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  h->mf_nharm = K;
  int rc = cg_phase<R>(h, nullptr, tol, max_iter);
  for (int k = 0; rc == CMCG_OK && k < K; ++k) {
    // filter weights of the frequency harm[k] w0 over T0, in the filtered sweep's table
    Prob Pk = P;
    Pk.omega = harm[k] * P.omega;
    filter_weights(Pk, s);
    std::vector<StageCoef<R>> tsf(static_cast<size_t>(h->L_srcf));
    for (int l = 0; l < h->L_srcf; ++l) {
      const int m = l / s, r = l % s;
      StageCoef<R> c;
      std::memset(&c, 0, sizeof(c));
      if (m < Pk.M || (m == Pk.M && r == 0)) {
        c.active = 1;
        source_coef<R>(s, r, Pk.dt, m * Pk.dt, Pk.omega, c);
        if (r == 0) {
          c.fa_re = R(Pk.fa[m].real());
          c.fa_im = R(Pk.fa[m].imag());
          c.fb_re = R(Pk.fb[m].real());
          c.fb_im = R(Pk.fb[m].imag());
        }
      }
      tsf[size_t(l)] = c;
    }
    CK(cudaMemcpyAsync(h->mf_tab, tsf.data(), tsf.size() * sizeof(StageCoef<R>), cudaMemcpyHostToDevice, h->stream));
    lincomb<R>(h, h->Uw, nullptr, nullptr, 1.0, h->U0, 0.0, nullptr);
    CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
    CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
    sweep_source<R>(h, true, true, nullptr);
    to_ext<R>(h, 0, h->Fre, 6, 0, e_re, 3, 3);
    to_ext<R>(h, 0, h->Fim, 6, 0, e_im, 3, 3);
    to_ext<R>(h, 0, h->Fre, 6, 3, h_re, 3, 3);
    to_ext<R>(h, 0, h->Fim, 6, 3, h_im, 3, 3);
    rc = sink(k);
    CK(cudaStreamSynchronize(h->stream));  // the host filter table is rebuilt for the next harmonic
  }
  h->mf_nharm = 0;
  if (rc) return rc;
  CK(cudaEventRecord(ev1, h->stream));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  if ((rc = check_err(h))) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, ev0, ev1);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return report(h, 1, tol, ms, K - 1, info);
}

// ------------------------------------------------------------------------------------------
// Slots: continuous batching on a batch handle.  Problem p is slot p; its phase is EMPTY,
// ADMITTED (source in place, Algorithm init pending), CG (iterating), FINAL (its CG stopped:
// filter pending) or DONE (result staged in ext0 / ext1 at the problem's offsets).  A round runs
// every phase's work with the problems of that phase masked in, in an order that keeps each
// problem's sequence of operations that of solve_dev: the source sweep of admitted slots, the
// forward sweep of iterating slots, one adjoint sweep for both, the CG updates of iterating
// slots, the reductions of Algorithm init for admitted slots (after the CG updates, which they
// must not take part in), and the filtered sweep of FINAL slots.
enum { SLOT_EMPTY = 0, SLOT_ADMITTED = 1, SLOT_CG = 2, SLOT_FINAL = 3, SLOT_DONE = 4 };

int slot_setup(cmcg_handle* h) {
  if (h->slot_masks) return CMCG_OK;
  if (cudaMalloc((void**)&h->slot_masks, sizeof(int32_t) * 3 * h->nprob) != cudaSuccess ||
      cudaMallocHost((void**)&h->slot_masks_host, sizeof(int32_t) * 3 * h->nprob) != cudaSuccess)
    return CMCG_ERR_OUT_OF_MEMORY;
  h->slot_phase.assign(size_t(h->nprob), SLOT_EMPTY);
  h->slot_info.assign(size_t(h->nprob), cmcg_info{});
  for (int p = 0; p < h->nprob; ++p) h->pactive_host[p] = 0;
  CK(cudaMemcpyAsync(h->pactive, h->pactive_host, sizeof(int32_t) * h->nprob, cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

template <typename R>
void zero_tiles(cmcg_handle* h, void* v, int p) {
  const Prob& P = h->P[size_t(p)];
  const size_t per_tile = size_t(6) * h->np * TILE * h->rsize;
  cudaMemsetAsync(static_cast<char*>(v) + size_t(P.tile0) * per_tile, 0, size_t(P.ntiles) * per_tile, h->stream);
}

template <typename R>
int slot_round_dev(cmcg_handle* h, double tol, int max_iter, int* done) {
  Range rg("cmcg: slot round");
  const int n = h->nprob;
  int32_t* mh = h->slot_masks_host;  // [admitted | adjoint | final]
  int32_t* m_init = h->slot_masks;
  int32_t* m_adj = h->slot_masks + n;
  int32_t* m_fin = h->slot_masks + 2 * n;
  bool any_init = false, any_cg = false, any_fin = false;
  for (int p = 0; p < n; ++p) {
    const int ph = h->slot_phase[size_t(p)];
    const bool cg = ph == SLOT_CG && h->pactive_host[p];
    mh[p] = ph == SLOT_ADMITTED;
    mh[n + p] = mh[p] || cg;
    mh[2 * n + p] = ph == SLOT_FINAL;
    any_init = any_init || mh[p];
    any_cg = any_cg || cg;
    any_fin = any_fin || mh[2 * n + p];
    if (done) done[p] = 0;
  }
  CK(cudaMemcpyAsync(h->slot_masks, mh, sizeof(int32_t) * 3 * n, cudaMemcpyHostToDevice, h->stream));
  if (any_init) {  // Algorithm init, first half: G = P_psi 0 (kept in A)
    for (int p = 0; p < n; ++p)
      if (mh[p]) {
        zero_tiles<R>(h, h->Uw, p);
        CK(cudaMemsetAsync(h->sc + p, 0, sizeof(Scalars), h->stream));
      }
    sweep_source<R>(h, true, false, m_init);
    launch_lincomb3_masked<R>((R*)h->A, nullptr, nullptr, 1.0, (const R*)h->Uw, 0.0, nullptr, h->nvec, h->np, h->tprob,
                              m_init, h->stream);
    h->launches++;
  }
  if (any_cg) {  // Algorithm grad on D: W_T = P D - D (iterating slots only: admitted slots hold G in Uw)
    sweep_free<R>(h, false, h->pactive);
    launch_lincomb3_masked<R>((R*)h->WT, (R*)h->Uw, nullptr, 1.0, (const R*)h->Uw, -1.0, (const R*)h->D, h->nvec,
                              h->np, h->tprob, h->pactive, h->stream);
    h->launches++;
  }
  if (any_init || any_cg) sweep_free<R>(h, true, m_adj);  // P* G (admitted), P* W_T (iterating)
  if (any_cg) {  // A = P* W_T - W_T and the CG update, as in solve_dev
    launch_cg_after_adjoint<R>(h->q, (const R*)h->Uw, (const R*)h->WT, (R*)h->A, (const R*)h->D, h->wdot, h->partials,
                               h->bt, h->pactive, h->stream);
    launch_finalize(h->partials, h->bt, h->sc, h->pactive, nullptr, 1, tol, h->stream);
    launch_cg_update<R>(h->q, (R*)h->U0, (R*)h->Rv, (const R*)h->D, (const R*)h->A, h->wdot, h->sc, h->partials, h->bt,
                        h->pactive, h->stream);
    launch_finalize(h->partials, h->bt, h->sc, h->pactive, nullptr, 2, tol, h->stream);
    launch_cg_direction<R>((R*)h->D, (R*)h->Uw, (const R*)h->Rv, h->sc, h->tprob, h->pactive, h->nvec, h->np,
                           h->stream);
    h->launches += 5;
  }
  if (any_init) {  // Algorithm init, second half: R = D = G* = G - P* G, U0 = 0, |R|^2
    launch_lincomb3_masked<R>((R*)h->Rv, (R*)h->D, (R*)h->Uw, 1.0, (const R*)h->A, -1.0, (const R*)h->Uw, h->nvec,
                              h->np, h->tprob, m_init, h->stream);
    for (int p = 0; p < n; ++p)
      if (mh[p]) zero_tiles<R>(h, h->U0, p);
    launch_dot<R>(h->q, (const R*)h->Rv, (const R*)h->Rv, h->wdot, h->partials, h->bt, h->stream);
    launch_finalize(h->partials, h->bt, h->sc, h->pactive, m_init, 4, tol, h->stream);
    h->launches += 3;
  }
  if (any_fin) {  // the final filter F_{psi,w} U0
    launch_lincomb3_masked<R>((R*)h->Uw, nullptr, nullptr, 1.0, (const R*)h->U0, 0.0, nullptr, h->nvec, h->np, h->tprob,
                              m_fin, h->stream);
    h->launches++;
    for (int p = 0; p < n; ++p)
      if (mh[2 * n + p]) {
        zero_tiles<R>(h, h->Fre, p);
        zero_tiles<R>(h, h->Fim, p);
      }
    sweep_source<R>(h, true, true, m_fin);
    const size_t half = size_t(h->nt_total) * 3 * h->np;
    for (int p = 0; p < n; ++p)
      if (mh[2 * n + p]) {
        const size_t off = size_t(h->P[size_t(p)].ext0) * 3 * h->np;
        to_ext<R>(h, p, h->Fre, 6, 0, h->ext0 + off, 3, 3);
        to_ext<R>(h, p, h->Fim, 6, 0, h->ext0 + half + off, 3, 3);
        to_ext<R>(h, p, h->Fre, 6, 3, h->ext1 + off, 3, 3);
        to_ext<R>(h, p, h->Fim, 6, 3, h->ext1 + half + off, 3, 3);
      }
  }
  CK(cudaGetLastError());
  int rc = read_state(h);
  if (rc) return rc;
  bool flip = false;
  for (int p = 0; p < n; ++p) {
    int& ph = h->slot_phase[size_t(p)];
    const Scalars& S = h->sc_host[p];
    if (ph == SLOT_FINAL) {
      int st = S.status;
      const bool conv = S.rr0 > 0 ? std::sqrt(std::max(S.rr, 0.0)) <= tol * std::sqrt(S.rr0) : true;
      if (st == CMCG_OK && !conv) st = CMCG_NOT_CONVERGED;
      cmcg_info& I = h->slot_info[size_t(p)];
      I = cmcg_info{};
      I.iters = S.iters;
      I.periods = 3 + 2 * S.iters;
      I.steps_per_period = h->P[size_t(p)].M;
      I.status = st;
      I.rel_residual = S.rr0 > 0 ? std::sqrt(std::max(S.rr, 0.0) / S.rr0) : 0.0;
      I.dt = h->P[size_t(p)].dt;
      ph = SLOT_DONE;
      if (done) done[p] = 1;
    } else if (ph == SLOT_ADMITTED) {
      ph = h->pactive_host[p] ? SLOT_CG : SLOT_FINAL;
    } else if (ph == SLOT_CG) {
      if (h->pactive_host[p] && S.iters >= max_iter) {  // stop at max_iter: the last iterate is filtered
        h->pactive_host[p] = 0;
        flip = true;
      }
      if (!h->pactive_host[p]) ph = SLOT_FINAL;
    }
  }
  if (flip) {
    CK(cudaMemcpyAsync(h->pactive, h->pactive_host, sizeof(int32_t) * n, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
  return CMCG_OK;
}

// Limiting amplitude ("full wave", Section 6): U = P_psi^periods 0, then
// F_psi U, for every problem of the handle.  The source is T-periodic, so the
// period map is affine, P_psi U = P U + G with G = P_psi 0: the march is one
// source sweep, then P U + G per further period (source-free sweeps; G kept in A).
template <typename R>
int fw_dev(cmcg_handle* h, int periods, const double* const* j_re, const double* const* j_im, double* const* e_re,
           double* const* e_im, double* const* h_re, double* const* h_im) {
  int rc = set_source<R>(h, j_re, j_im, h->nprob);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->Uw, 0, h->nvec * h->rsize, h->stream));
  if (periods > 0) sweep_source<R>(h, true, false, nullptr);
  if (periods > 1) lincomb<R>(h, h->A, nullptr, nullptr, 1.0, h->Uw, 0.0, nullptr);
  for (int l = 1; l < periods; ++l) {
    sweep_free<R>(h, false, nullptr);
    lincomb<R>(h, h->Uw, nullptr, nullptr, 1.0, h->Uw, 1.0, h->A);
  }
  CK(cudaMemsetAsync(h->Fre, 0, h->nvec * h->rsize, h->stream));
  CK(cudaMemsetAsync(h->Fim, 0, h->nvec * h->rsize, h->stream));
  sweep_source<R>(h, true, true, nullptr);
  for (int p = 0; p < h->nprob; ++p) {
    to_ext<R>(h, p, h->Fre, 6, 0, e_re[p], 3, 3);
    to_ext<R>(h, p, h->Fim, 6, 0, e_im[p], 3, 3);
    to_ext<R>(h, p, h->Fre, 6, 3, h_re[p], 3, 3);
    to_ext<R>(h, p, h->Fim, 6, 3, h_im[p], 3, 3);
  }
  CK(cudaGetLastError());
  return check_err(h);
}

// Forgets the captured sweep graphs (their launches embed the stage arguments); the next
// sweep of each kind is captured again.
void drop_graphs(cmcg_handle* h) {
  for (auto& kv : h->graph_exec) cudaGraphExecDestroy(kv.second);
  h->graph_exec.clear();
}

void free_all(cmcg_handle* h) {
  drop_graphs(h);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  h->cap_stream = nullptr;
  void* ptrs[] = {h->Jm_re, h->Jm_im, h->mf_hcs, h->mf_tab, h->mf_src,
                  h->gvol, h->gface, h->nbr, h->wdot, h->e_of_i, h->tprob, h->inv_eps, h->Uw, h->vA, h->vB,
                  h->Fre, h->Fim, h->Jre, h->Jim, h->Bre, h->Bim, h->U0, h->Rv, h->D, h->A, h->WT, h->partials, h->sc, h->pactive,
                  h->bt_tet0, h->bt_ntet, h->bt_prob, h->bt_pb0, h->tab_free, h->tab_src, h->tab_srcf, h->tab_one,
                  h->ext0, h->ext1, h->ext2, h->ext3, h->used, h->err, h->slot_masks, h->halo_dst, h->halo_src, h->g_in,
                  h->g_out, h->inv_eps_g};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->sc_host) cudaFreeHost(h->sc_host);
  if (h->pactive_host) cudaFreeHost(h->pactive_host);
  if (h->used_host) cudaFreeHost(h->used_host);
  if (h->err_host) cudaFreeHost(h->err_host);
  if (h->slot_masks_host) cudaFreeHost(h->slot_masks_host);
  for (auto& e : h->prof_ev) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
}

template <typename R>
std::vector<R> cast(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

template <typename T>
int upload(void** dst, const std::vector<T>& v, size_t* bytes) {
  const size_t n = std::max<size_t>(1, v.size()) * sizeof(T);
  CK(cudaMalloc(dst, n));
  if (!v.empty()) CK(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *bytes += n;
  return CMCG_OK;
}

int create_impl(int nprob, const cmcg_problem* probs, const cmcg_options* opt_in, cmcg_handle** out) {
  if (!out) return CMCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (nprob < 1 || !probs) return CMCG_ERR_INVALID_ARG;
  cmcg_options opt;
  if (opt_in) opt = *opt_in;
  else cmcg_default_options(&opt);
  cmcg_handle* h = new (std::nothrow) cmcg_handle();
  if (!h) return CMCG_ERR_OUT_OF_MEMORY;
  for (double& x : h->tune_us) x = -1;
  h->device = opt.device;
  h->q = opt.order;
  h->prec = opt.precision;
  h->s = opt.order == 1 ? 2 : 4;
  h->nprob = nprob;
  h->rsize = opt.precision == CMCG_FP32 ? 4 : 8;
  h->P.resize(nprob);
  // Host layouts, concatenated.
  std::vector<double> gvol, gface, wdot, inv_eps;
  std::vector<int32_t> nbr, e_of_i, tprob;
  int rc = CMCG_OK;
  try {
    for (int p = 0; p < nprob && rc == CMCG_OK; ++p) {
      HostLayout L;
      std::string why;
      rc = validate_and_layout(probs[p].mesh, probs[p].eps, probs[p].mu, probs[p].omega, &opt, &L, true, &why);
      if (rc) break;
      Prob& P = h->P[p];
      P.nt = L.nt;
      P.tet0 = h->nti;
      P.nti = L.nti;
      P.tile0 = h->ntiles;
      P.ntiles = L.ntiles;
      P.ext0 = h->nt_total;
      P.M = L.steps;
      P.dt = L.dt;
      P.T = L.T;
      P.omega = probs[p].omega;
      filter_weights(P, h->s);
      h->maxM = std::max(h->maxM, P.M);
      if (h->nti + L.nti > (int64_t(1) << 26)) {  // neighbour codes hold 26-bit internal indices
        rc = CMCG_ERR_INVALID_ARG;
        break;
      }
      gvol.insert(gvol.end(), L.gvol.begin(), L.gvol.end());
      gface.insert(gface.end(), L.gface.begin(), L.gface.end());
      wdot.insert(wdot.end(), L.wdot.begin(), L.wdot.end());
      const int32_t shift = int32_t(P.tet0) << 5;
      for (int32_t c : L.nbr) nbr.push_back(c >= 0 ? c + shift : c);
      for (int64_t t = 0; t < L.ntiles; ++t)
        for (int f = 0; f < 4; ++f)
          for (int l = 0; l < TILE; ++l) {
            if (L.nbr[(t * 4 + f) * TILE + l] != NBR_IMP || L.ext_of_int[t * TILE + l] < 0) continue;
            ImpFace F;
            F.it = P.tet0 + t * TILE + l;
            F.ext = L.ext_of_int[t * TILE + l];
            F.f = f;
            auto gf = [&](int item) { return L.gface[((t * 4 + f) * GF + item) * TILE + l]; };
            for (int a = 0; a < 3; ++a) F.n[a] = gf(a);
            F.bH = gf(3);
            F.aE = gf(6);
            P.imp.push_back(F);
          }
      e_of_i.insert(e_of_i.end(), L.ext_of_int.begin(), L.ext_of_int.end());
      P.ext_of_int = L.ext_of_int;
      P.int_of_ext = L.int_of_ext;
      for (int64_t t = 0; t < L.ntiles; ++t) tprob.push_back(p);
      for (int64_t k = 0; k < L.nt; ++k) inv_eps.push_back(1.0 / probs[p].eps[k]);
      h->nti += L.nti;
      h->ntiles += L.ntiles;
      h->nt_total += L.nt;
    }
  } catch (const std::bad_alloc&) {
    rc = CMCG_ERR_OUT_OF_MEMORY;
  } catch (...) {
    rc = CMCG_ERR_INVALID_ARG;
  }
  if (rc) {
    delete h;
    return rc;
  }
  h->np = np_of(h->q);
  h->nvec = h->nti * 6 * h->np;
  h->njvec = h->nti * 3 * h->np;
  // Problem-aligned reduction blocks.
  std::vector<int64_t> bt_tet0;
  std::vector<int32_t> bt_ntet, bt_prob, bt_pb0;
  for (int p = 0; p < nprob; ++p) {
    bt_pb0.push_back(int32_t(bt_tet0.size()));
    for (int64_t t = 0; t < h->P[p].nti; t += DOT_THREADS) {
      bt_tet0.push_back(h->P[p].tet0 + t);
      bt_ntet.push_back(int32_t(std::min<int64_t>(DOT_THREADS, h->P[p].nti - t)));
      bt_prob.push_back(p);
    }
  }
  bt_pb0.push_back(int32_t(bt_tet0.size()));

  const size_t extlen = size_t(h->nt_total) * 6 * h->np * sizeof(double);
  const size_t need = 11 * h->nvec * h->rsize + 2 * h->njvec * h->rsize + gvol.size() * h->rsize +
                      gface.size() * h->rsize + nbr.size() * 4 + wdot.size() * 8 + e_of_i.size() * 4 +
                      inv_eps.size() * 8 + 4 * extlen + bt_tet0.size() * 24 + size_t(nprob) * 128 +
                      size_t(3 * h->maxM * h->s + 2) * nprob * sizeof(StageCoef<double>);
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
  if (cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, opt.device) != cudaSuccess)
    return fail(CMCG_ERR_CUDA);

  size_t bytes = 0;
  if (h->prec == CMCG_FP32) {
    if ((rc = upload(&h->gvol, cast<float>(gvol), &bytes)) || (rc = upload(&h->gface, cast<float>(gface), &bytes)))
      return fail(rc);
  } else {
    if ((rc = upload(&h->gvol, gvol, &bytes)) || (rc = upload(&h->gface, gface, &bytes))) return fail(rc);
  }
  if ((rc = upload((void**)&h->nbr, nbr, &bytes)) || (rc = upload((void**)&h->wdot, wdot, &bytes)) ||
      (rc = upload((void**)&h->e_of_i, e_of_i, &bytes)) || (rc = upload((void**)&h->inv_eps, inv_eps, &bytes)) ||
      (rc = upload((void**)&h->bt_tet0, bt_tet0, &bytes)) || (rc = upload((void**)&h->bt_ntet, bt_ntet, &bytes)) ||
      (rc = upload((void**)&h->bt_prob, bt_prob, &bytes)) || (rc = upload((void**)&h->bt_pb0, bt_pb0, &bytes)))
    return fail(rc);
  if (nprob > 1 && (rc = upload((void**)&h->tprob, tprob, &bytes))) return fail(rc);
  h->bt = BlockTable{h->bt_tet0, h->bt_ntet, h->bt_prob, h->bt_pb0, int(bt_tet0.size()), nprob};

  auto alloc = [&](void** p, size_t n) -> bool { return cudaMalloc(p, n) == cudaSuccess; };
  const size_t vb = h->nvec * h->rsize, jb = h->njvec * h->rsize;
  bool ok = alloc(&h->Uw, vb) && alloc(&h->vA, vb) && alloc(&h->vB, vb) && alloc(&h->Fre, vb) &&
            alloc(&h->Fim, vb) && alloc(&h->Jre, jb) && alloc(&h->Jim, jb) && alloc(&h->U0, vb) &&
            alloc(&h->Rv, vb) && alloc(&h->D, vb) && alloc(&h->A, vb) && alloc(&h->WT, vb) &&
            alloc((void**)&h->partials, sizeof(double) * 2 * std::max<size_t>(1, bt_tet0.size())) &&
            alloc((void**)&h->sc, sizeof(Scalars) * nprob) && alloc((void**)&h->pactive, sizeof(int32_t) * nprob) &&
            alloc((void**)&h->used, sizeof(int32_t) * nprob) && alloc((void**)&h->err, sizeof(int32_t)) &&
            alloc((void**)&h->ext0, extlen) && alloc((void**)&h->ext1, extlen) && alloc((void**)&h->ext2, extlen) &&
            alloc((void**)&h->ext3, extlen);
  if (!ok) return fail(CMCG_ERR_OUT_OF_MEMORY);
  if (cudaMallocHost((void**)&h->sc_host, sizeof(Scalars) * nprob) != cudaSuccess ||
      cudaMallocHost((void**)&h->pactive_host, sizeof(int32_t) * nprob) != cudaSuccess ||
      cudaMallocHost((void**)&h->used_host, sizeof(int32_t) * nprob) != cudaSuccess ||
      cudaMallocHost((void**)&h->err_host, sizeof(int32_t)) != cudaSuccess)
    return fail(CMCG_ERR_OUT_OF_MEMORY);
  if (cudaMemset(h->err, 0, sizeof(int32_t)) != cudaSuccess)
    return fail(CMCG_ERR_CUDA);
  rc = h->prec == CMCG_FP32 ? build_tables<float>(h) : build_tables<double>(h);
  if (rc) return fail(rc);
  if (opt.stage_variant > 0) {
    const int nf = h->prec == CMCG_FP32 ? STAGE_FORMS_F32 : STAGE_FORMS_F64;
    if (opt.stage_variant > nf) return fail(CMCG_ERR_INVALID_ARG);
    h->form = opt.stage_variant - 1;
    h->pdl = opt.stage_overlap != 2;
  } else {
    rc = h->prec == CMCG_FP32 ? autotune<float>(h, STAGE_FORMS_F32, opt.stage_overlap)
                              : autotune<double>(h, STAGE_FORMS_F64, opt.stage_overlap);
    if (rc) return fail(rc);
  }
  h->graphs = opt.launch_graphs != 2;
  if (h->graphs && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    h->cap_stream = nullptr;
    h->graphs = false;
  }
  h->launches = 0;
  *out = h;
  return CMCG_OK;
}

bool single(const cmcg_handle* h) { return h && (h->nprob == 1 || h->coupled); }

// CMCG on a sharded handle: every part reads the global source and writes its owned results
// into the global outputs (device pointers); the report is the parts' common one.
int solve_sharded(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
                  double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  if (!j_re || !e_re || !e_im || !h_re || !h_im || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(h->nprob);
  std::vector<const double*> jr(n, j_re), ji(n, j_im);
  std::vector<double*> er(n, e_re), ei(n, e_im), hr(n, h_re), hi(n, h_im);
  std::vector<cmcg_info> infos(n);
  const int rc = h->prec == CMCG_FP32 ? solve_dev<float>(h, h->nprob, jr.data(), ji.data(), tol, max_iter, er.data(),
                                                         ei.data(), hr.data(), hi.data(), infos.data())
                                      : solve_dev<double>(h, h->nprob, jr.data(), ji.data(), tol, max_iter, er.data(),
                                                          ei.data(), hr.data(), hi.data(), infos.data());
  if (info) *info = infos[0];
  return rc;
}
bool batch_ok(const cmcg_handle* h) { return h && !h->coupled; }

}  // namespace

extern "C" {

void cmcg_default_options(cmcg_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->order = 1;
  opt->precision = CMCG_FP64;
  opt->flux = CMCG_FLUX_UPWIND;
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

int cmcg_create(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega, const cmcg_options* opt,
                cmcg_handle** out) {
  const cmcg_problem p{mesh, eps, mu, omega};
  return create_impl(1, &p, opt, out);
}

int cmcg_create_batch(int nprob, const cmcg_problem* probs, const cmcg_options* opt, cmcg_handle** out) {
  return create_impl(nprob, probs, opt, out);
}

int cmcg_create_sharded(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                        const cmcg_options* opt_in, int nparts, const int32_t* part, cmcg_handle** out) {
  if (!out) return CMCG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!mesh || !eps || !mu || !part || nparts < 1) return CMCG_ERR_INVALID_ARG;
  cmcg_options opt;
  if (opt_in) opt = *opt_in;
  else cmcg_default_options(&opt);
  // The global problem fixes M (Eq. cfl over all tetrahedra); every part steps with it.
  HostLayout G;
  std::string why;
  const size_t npt = static_cast<size_t>(nparts);
  std::vector<ShardPlan> plans(npt);
  std::vector<std::vector<int32_t>> tets(npt);
  std::vector<std::vector<double>> peps(npt), pmu(npt);
  std::vector<cmcg_mesh> meshes(npt);
  std::vector<cmcg_problem> probs(npt);
  try {
    int rc = validate_and_layout(mesh, eps, mu, omega, &opt, &G, false, &why);
    if (rc) return rc;
    if (nparts > mesh->nt) return CMCG_ERR_INVALID_ARG;
    for (int64_t k = 0; k < mesh->nt; ++k)
      if (part[k] < 0 || part[k] >= nparts) return CMCG_ERR_INVALID_ARG;
    std::vector<int64_t> nb;
    if (!match_faces(mesh, &nb)) return CMCG_ERR_NONCONFORMING_MESH;
    for (int p = 0; p < nparts; ++p) {
      if ((rc = shard_plan(mesh, nb, part, nparts, p, &plans[size_t(p)]))) return rc;
      const ShardPlan& S = plans[size_t(p)];
      if (S.n_owned == 0) return CMCG_ERR_INVALID_ARG;  // every part owns a tetrahedron
      for (int32_t k : S.global_of_local) {
        for (int v = 0; v < 4; ++v) tets[size_t(p)].push_back(mesh->tets[4 * int64_t(k) + v]);
        peps[size_t(p)].push_back(eps[k]);
        pmu[size_t(p)].push_back(mu[k]);
      }
      meshes[size_t(p)] = cmcg_mesh{mesh->nv, mesh->verts, int64_t(S.global_of_local.size()), tets[size_t(p)].data(),
                                    S.local_tags.data()};
      probs[size_t(p)] = cmcg_problem{&meshes[size_t(p)], peps[size_t(p)].data(), pmu[size_t(p)].data(), omega};
    }
  } catch (const std::bad_alloc&) {
    return CMCG_ERR_OUT_OF_MEMORY;
  }
  opt.steps_per_period = G.steps;
  cmcg_handle* h = nullptr;
  int rc = create_impl(nparts, probs.data(), &opt, &h);
  if (rc) return rc;
  auto fail = [&](int code) {
    cmcg_destroy(h);
    return code;
  };
  h->coupled = true;
  h->nt_global = mesh->nt;
  h->bt.coupled = 1;
  // Halo pairs (ghost <- owner) and the internal -> global maps.
  std::vector<int64_t> hdst, hsrc;
  std::vector<int32_t> gin(static_cast<size_t>(h->nti), -1), gout(static_cast<size_t>(h->nti), -1);
  for (int p = 0; p < nparts; ++p) {
    const ShardPlan& S = plans[size_t(p)];
    const Prob& P = h->P[size_t(p)];
    for (size_t g = 0; g < S.ghost_owner_part.size(); ++g) {
      const Prob& Q = h->P[size_t(S.ghost_owner_part[g])];
      hdst.push_back(P.tet0 + P.int_of_ext[size_t(S.n_owned) + g]);
      hsrc.push_back(Q.tet0 + Q.int_of_ext[size_t(S.ghost_owner_local[g])]);
    }
    for (int64_t i = 0; i < P.nti; ++i) {
      const int32_t e = P.ext_of_int[size_t(i)];
      if (e < 0) continue;
      gin[size_t(P.tet0 + i)] = S.global_of_local[size_t(e)];
      if (e < S.n_owned) gout[size_t(P.tet0 + i)] = S.global_of_local[size_t(e)];
    }
  }
  std::vector<double> ieg(static_cast<size_t>(mesh->nt));
  for (int64_t k = 0; k < mesh->nt; ++k) ieg[size_t(k)] = 1.0 / eps[k];
  size_t bytes = 0;
  if ((rc = upload((void**)&h->halo_dst, hdst, &bytes)) || (rc = upload((void**)&h->halo_src, hsrc, &bytes)) ||
      (rc = upload((void**)&h->g_in, gin, &bytes)) || (rc = upload((void**)&h->g_out, gout, &bytes)) ||
      (rc = upload((void**)&h->inv_eps_g, ieg, &bytes)))
    return fail(rc);
  h->bytes += bytes;
  h->nhalo = int64_t(hdst.size());
  // ghosts do not count in the inner products (their owners do)
  launch_zero_wdot(h->wdot, h->halo_dst, h->nhalo, h->stream);
  if (cudaStreamSynchronize(h->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(CMCG_ERR_CUDA);
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
  const int64_t n = h->coupled ? h->nt_global : h->P[0].nt;
  if (nt) *nt = n;
  if (np) *np = h->np;
  if (steps) *steps = h->P[0].M;
  if (dt) *dt = h->P[0].dt;
  if (field_len) *field_len = n * 6 * h->np;
  return CMCG_OK;
}

int cmcg_batch_size(const cmcg_handle* h) { return h ? h->nprob : 0; }

int cmcg_get_problem(const cmcg_handle* h, int p, int64_t* nt, int* steps, double* dt) {
  if (!h || p < 0 || p >= h->nprob) return CMCG_ERR_INVALID_ARG;
  if (nt) *nt = h->P[p].nt;
  if (steps) *steps = h->P[p].M;
  if (dt) *dt = h->P[p].dt;
  return CMCG_OK;
}

int64_t cmcg_kernel_launches(const cmcg_handle* h) { return h ? h->launches : 0; }

int cmcg_get_tuning(const cmcg_handle* h, int* variant, double* us_per_stage) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  if (variant) *variant = h->form;
  if (us_per_stage)
    for (int i = 0; i < 10; ++i) us_per_stage[i] = h->tune_us[i];
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
  if (!single(h) || !u || !out) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(ext_nt(h)) * 6 * h->np, nj = size_t(ext_nt(h)) * 3 * h->np;
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
  if (!single(h) || !u0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, forward_dev<float>(h, u0, j_re, j_im, uT, filt_re, filt_im),
                  forward_dev<double>(h, u0, j_re, j_im, uT, filt_re, filt_im));
}

int dgtd_period_adjoint_device(cmcg_handle* h, const double* wT, double* w0) {
  if (!single(h) || !wT || !w0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, adjoint_dev<float>(h, wT, w0), adjoint_dev<double>(h, wT, w0));
}

int dgtd_period_forward(cmcg_handle* h, const double* u0, const double* j_re, const double* j_im, double* uT,
                        double* filt_re, double* filt_im) {
  if (!single(h) || !u0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(ext_nt(h)) * 6 * h->np, nj = size_t(ext_nt(h)) * 3 * h->np;
  // ext0: u0 / uT, ext1: filter re, ext2: filter im, ext3: j (re, then im)
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
  int rc = DISPATCH(
      h, forward_dev<float>(h, h->ext0, jr, ji, h->ext0, filter ? h->ext1 : nullptr, filter ? h->ext2 : nullptr),
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
  if (!single(h) || !wT || !w0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(ext_nt(h)) * 6 * h->np;
  CK(cudaMemcpyAsync(h->ext0, wT, n * 8, cudaMemcpyHostToDevice, h->stream));
  int rc = DISPATCH(h, adjoint_dev<float>(h, h->ext0, h->ext0), adjoint_dev<double>(h, h->ext0, h->ext0));
  if (rc) return rc;
  CK(cudaMemcpyAsync(w0, h->ext0, n * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

int cmcg_inner(cmcg_handle* h, const double* u, const double* v, double* out) {
  if (!single(h) || !u || !v || !out) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t n = size_t(ext_nt(h)) * 6 * h->np;
  CK(cudaMemcpyAsync(h->ext0, u, n * 8, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->ext1, v, n * 8, cudaMemcpyHostToDevice, h->stream));
  return DISPATCH(h, inner_dev<float>(h, h->ext0, h->ext1, out), inner_dev<double>(h, h->ext0, h->ext1, out));
}

int cmcg_solve_batch_device(cmcg_handle* h, const double* const* j_re, const double* const* j_im, double tol,
                            int max_iter, double* const* e_re, double* const* e_im, double* const* h_re,
                            double* const* h_im, cmcg_info* info) {
  if (!batch_ok(h) || !j_re || !e_re || !e_im || !h_re || !h_im || !(tol >= 0) || max_iter < 0)
    return CMCG_ERR_INVALID_ARG;
  for (int p = 0; p < h->nprob; ++p)
    if (!j_re[p] || !e_re[p] || !e_im[p] || !h_re[p] || !h_im[p]) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  return DISPATCH(h, solve_dev<float>(h, h->nprob, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info),
                  solve_dev<double>(h, h->nprob, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info));
}

}  // extern "C"

namespace {

// Host-buffer entry points: sources copied into the staging vectors (ext3: all
// real parts, then all imaginary parts), results staged in ext0 (e) and ext1 (h).
struct HostIO {
  std::vector<const double*> jr, ji;
  std::vector<double*> er, ei, hr, hi;
};

int stage_host_inputs(cmcg_handle* h, int n, const double* const* j_re, const double* const* j_im, HostIO& io) {
  const size_t half = size_t(h->nt_total) * 3 * h->np;
  io.jr.assign(n, nullptr);
  io.ji.assign(n, nullptr);
  io.er.assign(n, nullptr);
  io.ei.assign(n, nullptr);
  io.hr.assign(n, nullptr);
  io.hi.assign(n, nullptr);
  for (int p = 0; p < n; ++p) {
    const size_t off = size_t(h->P[p].ext0) * 3 * h->np, cnt = size_t(h->P[p].nt) * 3 * h->np;
    CK(cudaMemcpyAsync(h->ext3 + off, j_re[p], cnt * 8, cudaMemcpyHostToDevice, h->stream));
    io.jr[p] = h->ext3 + off;
    if (j_im && j_im[p]) {
      CK(cudaMemcpyAsync(h->ext3 + half + off, j_im[p], cnt * 8, cudaMemcpyHostToDevice, h->stream));
      io.ji[p] = h->ext3 + half + off;
    }
    io.er[p] = h->ext0 + off;
    io.ei[p] = h->ext0 + half + off;
    io.hr[p] = h->ext1 + off;
    io.hi[p] = h->ext1 + half + off;
  }
  return CMCG_OK;
}

int copy_host_outputs(cmcg_handle* h, int n, const HostIO& io, double* const* e_re, double* const* e_im,
                      double* const* h_re, double* const* h_im) {
  for (int p = 0; p < n; ++p) {
    const size_t cnt = size_t(h->P[p].nt) * 3 * h->np;
    CK(cudaMemcpyAsync(e_re[p], io.er[p], cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(e_im[p], io.ei[p], cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h_re[p], io.hr[p], cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h_im[p], io.hi[p], cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  }
  CK(cudaStreamSynchronize(h->stream));
  return CMCG_OK;
}

bool host_args_ok(const cmcg_handle* h, int n, const double* const* j_re, double* const* e_re, double* const* e_im,
                  double* const* h_re, double* const* h_im) {
  if (!batch_ok(h) || n < 1 || n > h->nprob || !j_re || !e_re || !e_im || !h_re || !h_im) return false;
  for (int p = 0; p < n; ++p)
    if (!j_re[p] || !e_re[p] || !e_im[p] || !h_re[p] || !h_im[p]) return false;
  return true;
}

}  // namespace

extern "C" {

int cmcg_solve_batch_n(cmcg_handle* h, int n, const double* const* j_re, const double* const* j_im, double tol,
                       int max_iter, double* const* e_re, double* const* e_im, double* const* h_re,
                       double* const* h_im, cmcg_info* info) {
  if (!host_args_ok(h, n, j_re, e_re, e_im, h_re, h_im) || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  HostIO io;
  int rc = stage_host_inputs(h, n, j_re, j_im, io);
  if (rc) return rc;
  rc = DISPATCH(h,
                solve_dev<float>(h, n, io.jr.data(), io.ji.data(), tol, max_iter, io.er.data(), io.ei.data(),
                                 io.hr.data(), io.hi.data(), info),
                solve_dev<double>(h, n, io.jr.data(), io.ji.data(), tol, max_iter, io.er.data(), io.ei.data(),
                                  io.hr.data(), io.hi.data(), info));
  if (rc < 0) return rc;
  const int rc2 = copy_host_outputs(h, n, io, e_re, e_im, h_re, h_im);
  return rc2 ? rc2 : rc;
}

int cmcg_set_boundary_data(cmcg_handle* h, int problem, const double* g_re, const double* g_im) {
  if (!batch_ok(h) || problem < 0 || problem >= h->nprob) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  Prob& P = h->P[problem];
  const int np = h->np, nfp = nfp_of(h->q);
  const size_t R_ = h->rsize;
  const size_t off = size_t(P.tet0) * 6 * np, cnt = size_t(P.nti) * 6 * np;  // the problem's tiles
  if (!g_re) {  // clear
    if (h->Bre) {
      CK(cudaMemsetAsync(static_cast<char*>(h->Bre) + off * R_, 0, cnt * R_, h->stream));
      CK(cudaMemsetAsync(static_cast<char*>(h->Bim) + off * R_, 0, cnt * R_, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    P.has_bdata = false;
  } else {
    if (!h->Bre) {
      const size_t bytes = size_t(h->nvec) * R_;
      if (cudaMalloc(&h->Bre, bytes) != cudaSuccess) return CMCG_ERR_OUT_OF_MEMORY;
      if (cudaMalloc(&h->Bim, bytes) != cudaSuccess) {
        cudaFree(h->Bre);
        h->Bre = nullptr;
        return CMCG_ERR_OUT_OF_MEMORY;
      }
      h->bytes += 2 * bytes;
      CK(cudaMemsetAsync(h->Bre, 0, bytes, h->stream));
      CK(cudaMemsetAsync(h->Bim, 0, bytes, h->stream));
    }
    // The data term of Phi is linear in g: with the exterior state (g, 0) the flux of a face gains
    // aE (g - n (n.g)) on the E rows and bH n x g on the H rows, lifted like every flux.  Summed
    // here once per call in double precision for the tetrahedra with impedance faces only, then
    // scattered into the problem's zeroed rows.
    const RefMats& rm = ref_mats(h->q);
    const int rows = 6 * np;
    std::map<int64_t, int64_t> slot;  // internal tetrahedron -> compact row block
    for (const ImpFace& F : P.imp) slot.emplace(F.it, int64_t(slot.size()));
    std::vector<int64_t> tets(slot.size());
    for (const auto& kv : slot) tets[kv.second] = kv.first;
    std::vector<double> hre(tets.size() * rows, 0.0), him(tets.size() * rows, 0.0);
    for (const ImpFace& F : P.imp) {
      double* re = hre.data() + slot[F.it] * rows;
      double* im = him.data() + slot[F.it] * rows;
      for (int jf = 0; jf < nfp; ++jf) {
        double fE[2][3], fH[2][3];
        for (int part = 0; part < 2; ++part) {
          const double* g = part ? g_im : g_re;
          double gv[3] = {0, 0, 0};
          if (g)
            for (int c = 0; c < 3; ++c) gv[c] = g[((size_t(F.ext) * 4 + F.f) * 3 + c) * nfp + jf];
          const double ng = F.n[0] * gv[0] + F.n[1] * gv[1] + F.n[2] * gv[2];
          const double nxg[3] = {F.n[1] * gv[2] - F.n[2] * gv[1], F.n[2] * gv[0] - F.n[0] * gv[2],
                                 F.n[0] * gv[1] - F.n[1] * gv[0]};
          for (int c = 0; c < 3; ++c) {
            fE[part][c] = F.aE * (gv[c] - F.n[c] * ng);
            fH[part][c] = F.bH * nxg[c];
          }
        }
        for (int i = 0; i < np; ++i) {
          const double L = rm.LIFT[size_t(i) * 4 * nfp + F.f * nfp + jf];
          for (int c = 0; c < 3; ++c) {
            re[c * np + i] += L * fE[0][c];
            im[c * np + i] += L * fE[1][c];
            re[(3 + c) * np + i] += L * fH[0][c];
            im[(3 + c) * np + i] += L * fH[1][c];
          }
        }
      }
    }
    CK(cudaMemsetAsync(static_cast<char*>(h->Bre) + off * R_, 0, cnt * R_, h->stream));
    CK(cudaMemsetAsync(static_cast<char*>(h->Bim) + off * R_, 0, cnt * R_, h->stream));
    if (!tets.empty()) {
      double *dre = nullptr, *dim = nullptr;
      int64_t* dtet = nullptr;
      const size_t vb = hre.size() * sizeof(double);
      if (cudaMalloc(&dre, vb) != cudaSuccess || cudaMalloc(&dim, vb) != cudaSuccess ||
          cudaMalloc(&dtet, tets.size() * sizeof(int64_t)) != cudaSuccess) {
        cudaFree(dre);
        cudaFree(dim);
        cudaFree(dtet);
        return CMCG_ERR_OUT_OF_MEMORY;
      }
      cudaError_t e = cudaMemcpyAsync(dre, hre.data(), vb, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dim, him.data(), vb, cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(dtet, tets.data(), tets.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream);
      if (e == cudaSuccess) {
        if (h->prec == CMCG_FP32)
          launch_scatter_rows<float>((float*)h->Bre, (float*)h->Bim, dre, dim, dtet, int64_t(tets.size()), np,
                                     h->stream);
        else
          launch_scatter_rows<double>((double*)h->Bre, (double*)h->Bim, dre, dim, dtet, int64_t(tets.size()), np,
                                      h->stream);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);  // host buffers live until here
      cudaFree(dre);
      cudaFree(dim);
      cudaFree(dtet);
      if (e != cudaSuccess) return cuda_fail(e);
    } else {
      CK(cudaStreamSynchronize(h->stream));
    }
    P.has_bdata = true;
  }
  h->has_bdata = false;
  for (const Prob& Q : h->P) h->has_bdata = h->has_bdata || Q.has_bdata;
  return CMCG_OK;
}

int cmcg_set_conductivity(cmcg_handle* h, int problem, const double* sigma) {
  if (!batch_ok(h) || problem < 0 || problem >= h->nprob) return CMCG_ERR_INVALID_ARG;
  Prob& P = h->P[problem];
  const int s = h->s;
  // Real-axis stability of the explicit step: the damping -sigma/eps alone needs
  // dt sigma / eps within the RK interval (2 for RK2, about 2.78 for RK4); 2 is required.
  if (sigma) {
    std::vector<double> ie(static_cast<size_t>(P.nt));
    if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
    CK(cudaMemcpy(ie.data(), h->inv_eps + P.ext0, ie.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t k = 0; k < P.nt; ++k) {
      if (!(sigma[k] >= 0) || !std::isfinite(sigma[k])) return CMCG_ERR_INVALID_ARG;
      if (P.dt * sigma[k] * ie[size_t(k)] > 2.0) return CMCG_ERR_INVALID_ARG;
    }
  } else if (cudaSetDevice(h->device) != cudaSuccess) {
    return CMCG_ERR_CUDA;
  }
  (void)s;
  double* dsig = h->ext0;  // staging: nt_total * 6 Np doubles >= nt
  if (sigma) {
    CK(cudaMemcpyAsync(dsig, sigma, size_t(P.nt) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  } else {
    CK(cudaMemsetAsync(dsig, 0, size_t(P.nt) * sizeof(double), h->stream));
  }
  void* gv = static_cast<char*>(h->gvol) + size_t(P.tile0) * GV * TILE * h->rsize;
  if (h->prec == CMCG_FP32)
    launch_set_gvol_item<float>((float*)gv, 11, dsig, h->inv_eps + P.ext0, h->e_of_i + P.tet0, P.nti, h->stream);
  else
    launch_set_gvol_item<double>((double*)gv, 11, dsig, h->inv_eps + P.ext0, h->e_of_i + P.tet0, P.nti, h->stream);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));
  P.has_sigma = sigma != nullptr;
  bool any = false;
  for (const Prob& Q : h->P) any = any || Q.has_sigma;
  if (any != h->has_sigma) drop_graphs(h);
  h->has_sigma = any;
  return CMCG_OK;
}

int cmcg_fw_solve_batch(cmcg_handle* h, int periods, const double* const* j_re, const double* const* j_im,
                        double* const* e_re, double* const* e_im, double* const* h_re, double* const* h_im) {
  if (!host_args_ok(h, h ? h->nprob : 0, j_re, e_re, e_im, h_re, h_im) || periods < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  HostIO io;
  int rc = stage_host_inputs(h, h->nprob, j_re, j_im, io);
  if (rc) return rc;
  rc = DISPATCH(h,
                fw_dev<float>(h, periods, io.jr.data(), io.ji.data(), io.er.data(), io.ei.data(), io.hr.data(),
                              io.hi.data()),
                fw_dev<double>(h, periods, io.jr.data(), io.ji.data(), io.er.data(), io.ei.data(), io.hr.data(),
                               io.hi.data()));
  if (rc < 0) return rc;
  return copy_host_outputs(h, h->nprob, io, e_re, e_im, h_re, h_im);
}

int cmcg_fw_solve(cmcg_handle* h, const double* j_re, const double* j_im, int periods, double* e_re, double* e_im,
                  double* h_re, double* h_im) {
  if (!single(h)) return CMCG_ERR_INVALID_ARG;
  return cmcg_fw_solve_batch(h, periods, &j_re, &j_im, &e_re, &e_im, &h_re, &h_im);
}

int cmcg_solve_batch(cmcg_handle* h, const double* const* j_re, const double* const* j_im, double tol, int max_iter,
                     double* const* e_re, double* const* e_im, double* const* h_re, double* const* h_im,
                     cmcg_info* info) {
  if (!h) return CMCG_ERR_INVALID_ARG;
  return cmcg_solve_batch_n(h, h->nprob, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info);
}

int64_t cmcg_device_bytes(const cmcg_handle* h) { return h ? int64_t(h->bytes) : 0; }

int cmcg_slot_state(const cmcg_handle* h, int slot) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob) return CMCG_ERR_INVALID_ARG;
  return h->slot_phase.empty() ? SLOT_EMPTY : h->slot_phase[size_t(slot)];
}

int cmcg_slot_admit(cmcg_handle* h, int slot, const double* j_re, const double* j_im) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob || !j_re) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  int rc = slot_setup(h);
  if (rc) return rc;
  if (h->slot_phase[size_t(slot)] != SLOT_EMPTY) return CMCG_ERR_INVALID_ARG;
  const Prob& P = h->P[size_t(slot)];
  const size_t half = size_t(h->nt_total) * 3 * h->np;
  const size_t off = size_t(P.ext0) * 3 * h->np, cnt = size_t(P.nt) * 3 * h->np;
  const double* jr = h->ext3 + off;
  const double* ji = nullptr;
  CK(cudaMemcpyAsync(h->ext3 + off, j_re, cnt * 8, cudaMemcpyHostToDevice, h->stream));
  if (j_im) {
    CK(cudaMemcpyAsync(h->ext3 + half + off, j_im, cnt * 8, cudaMemcpyHostToDevice, h->stream));
    ji = h->ext3 + half + off;
  }
  if (h->prec == CMCG_FP32) {
    to_int<float>(h, slot, jr, 3, h->Jre, 3, 3, h->inv_eps);
    if (ji) to_int<float>(h, slot, ji, 3, h->Jim, 3, 3, h->inv_eps);
  } else {
    to_int<double>(h, slot, jr, 3, h->Jre, 3, 3, h->inv_eps);
    if (ji) to_int<double>(h, slot, ji, 3, h->Jim, 3, 3, h->inv_eps);
  }
  if (!ji) {
    const size_t per_tile = size_t(3) * h->np * TILE * h->rsize;
    CK(cudaMemsetAsync(static_cast<char*>(h->Jim) + size_t(P.tile0) * per_tile, 0, size_t(P.ntiles) * per_tile,
                       h->stream));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(h->stream));  // the host source may be reused when this returns
  h->slot_phase[size_t(slot)] = SLOT_ADMITTED;
  return CMCG_OK;
}

int cmcg_slot_round(cmcg_handle* h, double tol, int max_iter, int* done) {
  if (!h || h->coupled || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  int rc = slot_setup(h);
  if (rc) return rc;
  rc = DISPATCH(h, slot_round_dev<float>(h, tol, max_iter, done), slot_round_dev<double>(h, tol, max_iter, done));
  if (rc) return rc;
  return check_err(h);
}

int cmcg_slot_take(cmcg_handle* h, int slot, double* e_re, double* e_im, double* h_re, double* h_im,
                   cmcg_info* info) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob) return CMCG_ERR_INVALID_ARG;
  if (h->slot_phase.empty() || h->slot_phase[size_t(slot)] != SLOT_DONE) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const Prob& P = h->P[size_t(slot)];
  const size_t half = size_t(h->nt_total) * 3 * h->np;
  const size_t off = size_t(P.ext0) * 3 * h->np, cnt = size_t(P.nt) * 3 * h->np;
  if (e_re) CK(cudaMemcpyAsync(e_re, h->ext0 + off, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  if (e_im) CK(cudaMemcpyAsync(e_im, h->ext0 + half + off, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  if (h_re) CK(cudaMemcpyAsync(h_re, h->ext1 + off, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  if (h_im) CK(cudaMemcpyAsync(h_im, h->ext1 + half + off, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const cmcg_info& I = h->slot_info[size_t(slot)];
  if (info) *info = I;
  h->slot_phase[size_t(slot)] = SLOT_EMPTY;
  return I.status;
}

}  // extern "C"

namespace {

// Saved state of a slot (checkpoint between rounds): a header, then the problem's tiles of U0, R,
// D (6 Np values per tetrahedron each) and of the source J_re, J_im (3 Np each), in the handle's
// precision and internal layout.  Between rounds Uw holds D for an iterating slot; A and W_T are
// scratch of a round.  Restoring it gives the same bits as never having stopped.
struct SlotHeader {
  char magic[8];
  int32_t prec, q, np, M, phase, pactive;
  int64_t nt, ntiles;
  double dt, omega;
  Scalars sc;
};
constexpr char SLOT_MAGIC[8] = {'C', 'M', 'C', 'G', 'S', 'L', 'T', '1'};

size_t slot_payload(const cmcg_handle* h, int slot) {
  const Prob& P = h->P[size_t(slot)];
  return size_t(P.ntiles) * TILE * h->np * h->rsize * (3 * 6 + 2 * 3);
}

}  // namespace

extern "C" {

int64_t cmcg_slot_state_bytes(const cmcg_handle* h, int slot) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob) return CMCG_ERR_INVALID_ARG;
  return int64_t(sizeof(SlotHeader) + slot_payload(h, slot));
}

int cmcg_slot_save(cmcg_handle* h, int slot, void* buf, int64_t len) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob || !buf || len < cmcg_slot_state_bytes(h, slot))
    return CMCG_ERR_INVALID_ARG;
  if (h->slot_phase.empty()) return CMCG_ERR_INVALID_ARG;
  const int ph = h->slot_phase[size_t(slot)];
  if (ph != SLOT_ADMITTED && ph != SLOT_CG && ph != SLOT_FINAL) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const Prob& P = h->P[size_t(slot)];
  SlotHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, SLOT_MAGIC, 8);
  hd.prec = h->prec;
  hd.q = h->q;
  hd.np = h->np;
  hd.M = P.M;
  hd.phase = ph;
  hd.nt = P.nt;
  hd.ntiles = P.ntiles;
  hd.dt = P.dt;
  hd.omega = P.omega;
  CK(cudaMemcpyAsync(&hd.sc, h->sc + slot, sizeof(Scalars), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&hd.pactive, h->pactive + slot, sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream));
  char* out = static_cast<char*>(buf) + sizeof(SlotHeader);
  const size_t v6 = size_t(P.ntiles) * 6 * h->np * TILE * h->rsize, v3 = v6 / 2;
  const size_t o6 = size_t(P.tile0) * 6 * h->np * TILE * h->rsize, o3 = o6 / 2;
  const void* src6[3] = {h->U0, h->Rv, h->D};
  for (int k = 0; k < 3; ++k, out += v6)
    CK(cudaMemcpyAsync(out, static_cast<const char*>(src6[k]) + o6, v6, cudaMemcpyDeviceToHost, h->stream));
  const void* src3[2] = {h->Jre, h->Jim};
  for (int k = 0; k < 2; ++k, out += v3)
    CK(cudaMemcpyAsync(out, static_cast<const char*>(src3[k]) + o3, v3, cudaMemcpyDeviceToHost, h->stream));
  const int32_t zero = 0;
  CK(cudaMemcpyAsync(h->pactive + slot, &zero, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  std::memcpy(buf, &hd, sizeof(hd));
  h->pactive_host[slot] = 0;
  h->slot_phase[size_t(slot)] = SLOT_EMPTY;
  return CMCG_OK;
}

int cmcg_slot_restore(cmcg_handle* h, int slot, const void* buf, int64_t len) {
  if (!h || h->coupled || slot < 0 || slot >= h->nprob || !buf || len < int64_t(sizeof(SlotHeader)))
    return CMCG_ERR_INVALID_ARG;
  SlotHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  const Prob& P = h->P[size_t(slot)];
  if (std::memcmp(hd.magic, SLOT_MAGIC, 8) != 0 || hd.prec != h->prec || hd.q != h->q || hd.np != h->np ||
      hd.M != P.M || hd.nt != P.nt || hd.ntiles != P.ntiles || hd.dt != P.dt || hd.omega != P.omega ||
      (hd.phase != SLOT_ADMITTED && hd.phase != SLOT_CG && hd.phase != SLOT_FINAL) ||
      len < int64_t(sizeof(SlotHeader) + slot_payload(h, slot)))
    return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  int rc = slot_setup(h);
  if (rc) return rc;
  if (h->slot_phase[size_t(slot)] != SLOT_EMPTY) return CMCG_ERR_INVALID_ARG;
  const char* in = static_cast<const char*>(buf) + sizeof(SlotHeader);
  const size_t v6 = size_t(P.ntiles) * 6 * h->np * TILE * h->rsize, v3 = v6 / 2;
  const size_t o6 = size_t(P.tile0) * 6 * h->np * TILE * h->rsize, o3 = o6 / 2;
  void* dst6[3] = {h->U0, h->Rv, h->D};
  for (int k = 0; k < 3; ++k, in += v6)
    CK(cudaMemcpyAsync(static_cast<char*>(dst6[k]) + o6, in, v6, cudaMemcpyHostToDevice, h->stream));
  void* dst3[2] = {h->Jre, h->Jim};
  for (int k = 0; k < 2; ++k, in += v3)
    CK(cudaMemcpyAsync(static_cast<char*>(dst3[k]) + o3, in, v3, cudaMemcpyHostToDevice, h->stream));
  // an iterating slot starts its next round with Uw = D
  CK(cudaMemcpyAsync(static_cast<char*>(h->Uw) + o6, static_cast<const char*>(h->D) + o6, v6,
                     cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(h->sc + slot, &hd.sc, sizeof(Scalars), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->pactive + slot, &hd.pactive, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->pactive_host[slot] = hd.pactive;
  h->slot_phase[size_t(slot)] = hd.phase;
  return CMCG_OK;
}

int cmcg_solve_multifreq(cmcg_handle* h, int nharm, const int* harmonics, const double* const* j_re,
                         const double* const* j_im, double tol, int max_iter, double* const* e_re,
                         double* const* e_im, double* const* h_re, double* const* h_im, cmcg_info* info) {
  if (!h || h->nprob != 1 || h->coupled || nharm < 1 || nharm > 64 || !harmonics || !j_re || !e_re || !e_im ||
      !h_re || !h_im || !(tol >= 0) || max_iter < 0)
    return CMCG_ERR_INVALID_ARG;
  for (int k = 0; k < nharm; ++k)
    if (harmonics[k] < 1 || !j_re[k] || !e_re[k] || !e_im[k] || !h_re[k] || !h_im[k]) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  const size_t nj = size_t(h->nt_total) * 3 * h->np;
  // the host sources go to a device buffer of 2 nharm sources, kept for later calls
  const size_t need = 2 * size_t(nharm) * nj;
  if (need > h->mf_src_len) {
    if (h->mf_src) cudaFree(h->mf_src);
    h->mf_src = nullptr;
    h->mf_src_len = 0;
    if (cudaMalloc((void**)&h->mf_src, need * sizeof(double)) != cudaSuccess) return CMCG_ERR_OUT_OF_MEMORY;
    h->mf_src_len = need;
    h->bytes += need * sizeof(double);
  }
  std::vector<const double*> djr(static_cast<size_t>(nharm)), dji(static_cast<size_t>(nharm), nullptr);
  for (int k = 0; k < nharm; ++k) {
    double* re = h->mf_src + 2 * size_t(k) * nj;
    CK(cudaMemcpyAsync(re, j_re[k], nj * 8, cudaMemcpyHostToDevice, h->stream));
    djr[size_t(k)] = re;
    if (j_im && j_im[k]) {
      CK(cudaMemcpyAsync(re + nj, j_im[k], nj * 8, cudaMemcpyHostToDevice, h->stream));
      dji[size_t(k)] = re + nj;
    }
  }
  // results of each harmonic through the staging vectors: e in ext0 (re, im), h in ext1
  double *de_re = h->ext0, *de_im = h->ext0 + nj, *dh_re = h->ext1, *dh_im = h->ext1 + nj;
  auto sink = [&](int k) -> int {
    CK(cudaMemcpyAsync(e_re[k], de_re, nj * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(e_im[k], de_im, nj * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h_re[k], dh_re, nj * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(h_im[k], dh_im, nj * 8, cudaMemcpyDeviceToHost, h->stream));
    return CMCG_OK;
  };
  return DISPATCH(h,
                  solve_multi_dev<float>(h, nharm, harmonics, djr.data(), dji.data(), tol, max_iter, de_re, de_im,
                                         dh_re, dh_im, sink, info),
                  solve_multi_dev<double>(h, nharm, harmonics, djr.data(), dji.data(), tol, max_iter, de_re, de_im,
                                          dh_re, dh_im, sink, info));
}

int cmcg_solve_device(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
                      double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  if (!single(h)) return CMCG_ERR_INVALID_ARG;
  if (!h->coupled) return cmcg_solve_batch_device(h, &j_re, &j_im, tol, max_iter, &e_re, &e_im, &h_re, &h_im, info);
  return solve_sharded(h, j_re, j_im, tol, max_iter, e_re, e_im, h_re, h_im, info);
}

int cmcg_solve(cmcg_handle* h, const double* j_re, const double* j_im, double tol, int max_iter, double* e_re,
               double* e_im, double* h_re, double* h_im, cmcg_info* info) {
  if (!single(h)) return CMCG_ERR_INVALID_ARG;
  if (!h->coupled) return cmcg_solve_batch(h, &j_re, &j_im, tol, max_iter, &e_re, &e_im, &h_re, &h_im, info);
  if (!j_re || !e_re || !e_im || !h_re || !h_im || !(tol >= 0) || max_iter < 0) return CMCG_ERR_INVALID_ARG;
  if (cudaSetDevice(h->device) != cudaSuccess) return CMCG_ERR_CUDA;
  // global source into ext3 (re, then im), results into ext0 (e) and ext1 (h)
  const size_t nj = size_t(h->nt_global) * 3 * h->np;
  CK(cudaMemcpyAsync(h->ext3, j_re, nj * 8, cudaMemcpyHostToDevice, h->stream));
  const double* ji = nullptr;
  if (j_im) {
    CK(cudaMemcpyAsync(h->ext3 + nj, j_im, nj * 8, cudaMemcpyHostToDevice, h->stream));
    ji = h->ext3 + nj;
  }
  int rc = solve_sharded(h, h->ext3, ji, tol, max_iter, h->ext0, h->ext0 + nj, h->ext1, h->ext1 + nj, info);
  if (rc < 0) return rc;
  CK(cudaMemcpyAsync(e_re, h->ext0, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(e_im, h->ext0 + nj, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h_re, h->ext1, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h_im, h->ext1 + nj, nj * 8, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return rc;
}

}  // extern "C"
