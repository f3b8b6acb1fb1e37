// One explicit Runge-Kutta stage of the DG time-domain Maxwell scheme, for a
// fixed polynomial order CMCG_Q (included once per order by dg_q{1,2,3}.cu).
//
// Two threads (adjacent lanes) share one tetrahedron K.  The even lane holds
// the electric field of K and computes Phi_H, the odd lane holds the magnetic
// field and computes Phi_E:
//
//   Phi_H =  mu^{-1} curl E + LIFT . fH,    Phi_E = -eps^{-1} curl H + LIFT . fE
//
// (Eq. ode_system: Phi(t, U) = Re(J e^{i w t}) + B U, strong form of the 3D
// upwind DG operator generalising Eq. DG_semidiscrete).  The curl of a thread's
// own field is all its volume term needs, so the volume work is not
// duplicated.  Face terms use jumps dE = E^+ - E^-, dH = H^+ - H^-; each thread
// forms the jump of its own field (neighbour trace, or the PEC mirror state
// dE = -2 E^-, dH = 0, or the impedance zero state dE = -E^-, dH = -H^-) and the
// partner's jump arrives by one lane shuffle per component.  With X its own jump
// and Y the partner's,
//
//   f = k1 (n x X) + k2 (Y - n (n . Y)),
//   (k1, k2) = (bH, aH) on the E lane  ->  fH = bH n x dE + aH dH_t,
//   (k1, k2) = (-bE, aE) on the H lane ->  fE = aE dE_t - bE n x dH,
//   aE = fscale / (eps (Z^- + Z^+)), bE = Z^+ aE, aH = fscale / (mu (Y^- + Y^+)), bH = Y^+ aH,
//
// which is -n x (H^ - H^-) and n x (E^ - E^-) for the upwind traces
// E^ = (Y^- E^- + Y^+ E^+ - (H^- - H^+) x n) / (Y^- + Y^+),
// H^ = (Z^- H^- + Z^+ H^+ + (E^- - E^+) x n) / (Z^- + Z^+);
// fscale = |F| / (|F_ref| |det A|) folds the block-diagonal inverse mass into
// the lift.  The adjoint stage (Section 4.1.2, P* = Sigma P Sigma) flips the
// sign of every magnetic value read and of Phi_H (sH = -1): no memory pass.
//
// Reference matrices D_r, D_s, D_t and LIFT live in constant memory; with the
// loops unrolled their indices are compile-time constants, so they are read as
// constant-bank operands of the FMAs.  A thread's neighbour traces (3 components
// x Nfp nodes x 4 faces) are copied into shared memory with cp.async before the
// volume loop, so their latency overlaps the curl computation; every thread
// reads back only the slots it filled (slot-major layout, conflict-free).
#pragma once

#include <cstring>

#include "common.h"

#ifndef CMCG_Q
#error "define CMCG_Q before including dg_stage.cuh"
#endif

namespace cmcg {
namespace {

constexpr int NPQ = np_of(CMCG_Q);
constexpr int NFPQ = nfp_of(CMCG_Q);

__constant__ float cDf[3 * NPQ * NPQ];
__constant__ double cDd[3 * NPQ * NPQ];
__constant__ float cLf[NPQ * 4 * NFPQ];
__constant__ double cLd[NPQ * 4 * NFPQ];
__constant__ signed char cNB[4 * 6 * NFPQ];

template <typename R>
__device__ __forceinline__ R cD(int idx) {
  if constexpr (sizeof(R) == 4) return cDf[idx];
  else return cDd[idx];
}
template <typename R>
__device__ __forceinline__ R cL(int idx) {
  if constexpr (sizeof(R) == 4) return cLf[idx];
  else return cLd[idx];
}

constexpr int STAGE_THREADS = 128;
constexpr int TRACE_SLOTS = 4 * NFPQ * 3;  // per thread

__device__ __forceinline__ void cp_async_4(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
// Programmatic dependent launch: a stage may be launched while the previous
// stage is still running (once all its blocks are resident); before
// grid_dep_wait(), which returns once the previous grid has completed and its
// writes are visible, it reads only data that no kernel writes (geometry,
// neighbour codes, face coefficients, coefficient tables, tile problems).
// Without the launch attribute both are no-ops.
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// The source on the E rows, added by the thread that computes Phi_E (Eq. ode_system): at the
// stage time, Re(J e^{i w t}) = s_cos J_re - s_sin J_im, or, in a sweep driven at several
// harmonics of a base frequency (a.nharm > 0), the sum over the harmonics of
// hcs[2h] J_re,h - hcs[2h+1] J_im,h.  Output nodes n0 .. n0 + NN - 1 of (tile, lane).
template <typename R, int NN>
__device__ __forceinline__ void add_source(R (&phi)[3][NN], const StageArgs<R>& a, const StageCoef<R>& cf,
                                           int64_t tile, int lane, int n0) {
  constexpr int NP = NPQ;
  const int64_t joff = tile * (3 * NP * TILE) + lane;
  if (a.nharm <= 0) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NN; ++ii) {
        const int64_t o = joff + (c * NP + n0 + ii) * TILE;
        phi[c][ii] += cf.s_cos * a.jre[o] - cf.s_sin * a.jim[o];
      }
    return;
  }
#pragma unroll 1
  for (int hh = 0; hh < a.nharm; ++hh) {
    const R sc = a.hcs[2 * hh], ss = a.hcs[2 * hh + 1];
    const R* jr = a.jre + hh * a.jstride;
    const R* ji = a.jim + hh * a.jstride;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NN; ++ii) {
        const int64_t o = joff + (c * NP + n0 + ii) * TILE;
        phi[c][ii] += sc * jr[o] - ss * ji[o];
      }
  }
}

// The on-the-fly filter on this thread's output rows n0 .. n0 + NN - 1 (forward sweeps with the
// filter, first nested stage of each step): F += fa U + fb Phi.  Each component's rows of U and F
// are loaded before any of them is stored: vin, fre and fim are not known to be distinct, and a
// row-by-row read-modify-write would put every load behind the previous row's stores.
template <typename R, int NN>
__device__ __forceinline__ void accumulate_filter(const StageArgs<R>& a, const StageCoef<R>& cf,
                                                  const R (&phi)[3][NN], int64_t off, int n0) {
  constexpr int NP = NPQ;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    R u[NN], fr[NN], fi[NN];
#pragma unroll
    for (int ii = 0; ii < NN; ++ii) {
      const int64_t o = off + (c * NP + n0 + ii) * TILE;
      u[ii] = a.vin[o];
      fr[ii] = a.fre[o];
      fi[ii] = a.fim[o];
    }
#pragma unroll
    for (int ii = 0; ii < NN; ++ii) {
      const int64_t o = off + (c * NP + n0 + ii) * TILE;
      a.fre[o] = fr[ii] + (cf.fa_re * u[ii] + cf.fb_re * phi[c][ii]);
      a.fim[o] = fi[ii] + (cf.fa_im * u[ii] + cf.fb_im * phi[c][ii]);
    }
  }
}

// MINB: minimum resident blocks per SM requested from the compiler (caps registers at
// 65536 / (MINB * STAGE_THREADS)); the forms are timed per handle (see api.cu).
template <typename R, int MINB>
__global__ void __launch_bounds__(STAGE_THREADS, MINB) dg_stage_kernel(const StageArgs<R> a) {
  constexpr int NP = NPQ, NFP = NFPQ;
  constexpr int VS = 6 * NP * TILE;  // elements per tile of a field vector
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  grid_dep_launch();
  const int64_t gthr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gt = gthr >> 1;  // tetrahedron; nti is a multiple of 32, so whole warps leave together
  if (gt >= a.nti) return;
  const int half = int(gthr & 1);  // 0: owns E, computes Phi_H;  1: owns H, computes Phi_E
  const int64_t tile = gt >> 5;
  const int lane = int(gt & 31);
  // A warp (16 tetrahedra) lies inside one tile, hence inside one problem: uniform exits.
  const int prob = a.tprob ? a.tprob[tile] : 0;
  const StageCoef<R> cf = a.coef[prob];
  if (!cf.active) return;
  const int cOwn = half ? 3 : 0, cOut = half ? 0 : 3;
  const R sH = a.sH;
  const R sIn = half ? sH : R(1);   // sign of the own field (magnetic values flipped in the adjoint)
  const R sOut = half ? R(1) : sH;  // sign of Phi_H
  const R pec = half ? R(0) : R(-2);  // PEC mirror: dE = -2 E^-, dH = 0

  // Loads of data no stage writes first (affine factors, codes, face coefficients),
  // then, once the previous stage is complete, the own field, the base rows and the
  // neighbour traces into shared memory (their addresses need the codes).
  R G[9];
  const R* gv = a.gvol + tile * GV * TILE + lane;
#pragma unroll
  for (int m = 0; m < 9; ++m) G[m] = gv[m * TILE];
  const R sv = half ? -gv[9 * TILE] : gv[10 * TILE] * sOut;  // -1/eps for Phi_E, sH/mu for Phi_H
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* tr = reinterpret_cast<R*>(smem_raw) + threadIdx.x;  // slot k at tr[k * STAGE_THREADS]
  int32_t code[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) code[f] = a.nbr[(tile * 4 + f) * TILE + lane];
  R fn[4][3], fk1[4], fk2[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const R* gf = a.gface + (tile * 4 + f) * GF * TILE + lane;
    fn[f][0] = gf[0];
    fn[f][1] = gf[TILE];
    fn[f][2] = gf[2 * TILE];
    fk1[f] = gf[(3 + 2 * half) * TILE] * sOut;
    fk2[f] = gf[(4 + 2 * half) * TILE] * sOut;
  }
  grid_dep_wait();
  if (a.pactive && !a.pactive[prob]) return;  // CG converged for this problem (written by the CG kernels)
  R v[3][NP];
  {
    const R* vin = a.vin + tile * VS + cOwn * NP * TILE + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) v[c][n] = sIn * vin[(c * NP + n) * TILE];
  }
  const int64_t off = tile * VS + cOut * NP * TILE + lane;
  R bv[3][NP];
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) bv[c][n] = a.base[off + (c * NP + n) * TILE];
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    if (code[f] >= 0) {
      const int64_t k = int64_t(code[f] >> 5);
      const R* nb = a.vin + (k >> 5) * VS + cOwn * NP * TILE + (k & 31);
      const int tab = (((code[f] >> 3) & 3) * 6 + (code[f] & 7)) * NFP;
#pragma unroll
      for (int jf = 0; jf < NFP; ++jf) {
        const int nn = cNB[tab + jf];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          R* dst = tr + ((f * NFP + jf) * 3 + c) * STAGE_THREADS;
          if constexpr (sizeof(R) == 4) cp_async_4(dst, nb + (c * NP + nn) * TILE);
          else cp_async_8(dst, nb + (c * NP + nn) * TILE);
        }
      }
    }
  }
  // Single-frequency source stages: the tetrahedron's source rows, J_re by the lane that adds
  // the source (half = 1) and J_im by its partner, fetched now so that their latency overlaps
  // the volume and face work.
  R* js = tr + TRACE_SLOTS * STAGE_THREADS;
  const bool jpre = a.jre && a.nharm <= 0;
  if (jpre) {
    const R* src = (half ? a.jre : a.jim) + tile * (3 * NP * TILE) + lane;
#pragma unroll
    for (int k = 0; k < 3 * NP; ++k) {
      if constexpr (sizeof(R) == 4) cp_async_4(js + k * STAGE_THREADS, src + k * TILE);
      else cp_async_8(js + k * STAGE_THREADS, src + k * TILE);
    }
  }
  cp_async_commit();

  R phi[3][NP];
  {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R d[3][3];
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[b][c] = R(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const R dr = cD<R>((0 * NP + i) * NP + j), ds = cD<R>((1 * NP + i) * NP + j), dt = cD<R>((2 * NP + i) * NP + j);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          d[0][c] = fma(dr, v[c][j], d[0][c]);
          d[1][c] = fma(ds, v[c][j], d[1][c]);
          d[2][c] = fma(dt, v[c][j], d[2][c]);
        }
      }
      // d/dx_ax of component c = sum_b G[b][ax] d[b][c]
      auto dx = [&](int ax, int c) { return G[0 * 3 + ax] * d[0][c] + G[1 * 3 + ax] * d[1][c] + G[2 * 3 + ax] * d[2][c]; };
      phi[0][i] = sv * (dx(1, 2) - dx(2, 1));
      phi[1][i] = sv * (dx(2, 0) - dx(0, 2));
      phi[2][i] = sv * (dx(0, 1) - dx(1, 0));
    }
  }

  cp_async_wait_all();
  __syncwarp();  // the partner's prefetched source rows are read at the end
  // The face term in two passes: first every face node's flux (24 independent
  // chains of trace read, jump, partner shuffle and flux, stored over the trace
  // slots the thread owns), then the lift as a stream of FMAs.  The values and
  // the order of the lift sums are those of a single pass.
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const R n0 = fn[f][0], n1 = fn[f][1], n2 = fn[f][2];
    const R k1 = fk1[f], k2 = fk2[f];
    const bool interior = code[f] >= 0;
    const R bscale = code[f] == NBR_PEC ? pec : R(-1);  // boundary jump = bscale * own trace
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      const int own = FM.v[f][jf];
      R X[3], Y[3];
      if (interior) {
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = sIn * tr[((f * NFP + jf) * 3 + c) * STAGE_THREADS] - v[c][own];
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = bscale * v[c][own];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[c] = __shfl_xor_sync(0xffffffffu, X[c], 1);
      const R nY = n0 * Y[0] + n1 * Y[1] + n2 * Y[2];
      tr[((f * NFP + jf) * 3 + 0) * STAGE_THREADS] = k1 * (n1 * X[2] - n2 * X[1]) + k2 * (Y[0] - n0 * nY);
      tr[((f * NFP + jf) * 3 + 1) * STAGE_THREADS] = k1 * (n2 * X[0] - n0 * X[2]) + k2 * (Y[1] - n1 * nY);
      tr[((f * NFP + jf) * 3 + 2) * STAGE_THREADS] = k1 * (n0 * X[1] - n1 * X[0]) + k2 * (Y[2] - n2 * nY);
    }
  }
  // pass 2: the lift
#pragma unroll
  for (int f = 0; f < 4; ++f) {
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      R fl[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) fl[c] = tr[((f * NFP + jf) * 3 + c) * STAGE_THREADS];
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const R L = cL<R>(i * 4 * NFP + f * NFP + jf);
#pragma unroll
        for (int c = 0; c < 3; ++c) phi[c][i] = fma(L, fl[c], phi[c][i]);
      }
    }
  }

  if (half && a.sigma) {  // conductivity: Phi_E -= (sigma / eps) E (E is not flipped by Sigma)
    const R so = a.gvol[(tile * GV + 11) * TILE + lane];
    const R* ev = a.vin + tile * VS + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) phi[c][n] -= so * ev[(c * NP + n) * TILE];
  }
  if (half && jpre) {  // source on the E rows: J_re in this thread's slots, J_im in the partner's
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int k = (c * NP + n) * STAGE_THREADS;
        phi[c][n] += cf.s_cos * js[k] - cf.s_sin * js[k - 1];
      }
  } else if (half && a.jre) {
    add_source<R, NP>(phi, a, cf, tile, lane, 0);
  }
  if (a.bre) {  // impedance-face data, lifted onto this thread's output rows (source sweeps only)
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        phi[c][n] += cf.s_cos * a.bre[o] - cf.s_sin * a.bim[o];
      }
  }
  if (a.fre) accumulate_filter<R, NP>(a, cf, phi, off, 0);  // forward sweeps with the filter only
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        a.out[o] = bv[c][n] + cf.c_out * phi[c][n];
      }
  }
}

// Four threads per tetrahedron: (E | H) x (node half).  A block of 128
// threads is one 32-tetrahedron tile.  Warps 2g and 2g + 1 share tetrahedra
// 16g .. 16g + 15 of the tile; in both, lanes (2t, 2t + 1) hold the electric
// and the magnetic field of tetrahedron 16g + t (roles as in dg_stage_kernel).
// Warp 2g + p computes the output rows of the nodes [p NH, p NH + NH) and the
// fluxes of faces 2p and 2p + 1: it lifts its own faces' fluxes onto its
// nodes, leaves them in shared memory for warp 2g + (1 - p), and after a
// barrier of the block lifts that warp's fluxes.  The arithmetic per output
// value (volume sums over j, lift sums over faces and face nodes) follows the
// same order as dg_stage_kernel.  p is warp-uniform, so the reference-matrix
// entries stay compile-time constant-bank operands; per thread the state is
// the own field (3 Np), half of the output rows and two faces, which leaves
// room for more resident warps.
constexpr int QD_THREADS = 128;
constexpr int QD_NH = NPQ / 2;                 // output nodes per thread
constexpr int QD_FSLOTS = 2 * NFPQ * 3;        // per thread: two faces x Nfp x 3 components
constexpr int QD_BSLOTS = 3 * QD_NH;           // per thread: base rows of its nodes

template <typename R>
constexpr size_t quad_smem() {
  return size_t(QD_THREADS) * (2 * QD_FSLOTS + QD_BSLOTS) * sizeof(R);
}

// Barrier of the 128 threads of the block (named barrier 1; every warp reaches
// it from its own half's code path).
__device__ __forceinline__ void quad_barrier() { asm volatile("bar.sync 1, 128;\n" ::: "memory"); }

template <typename R, int P>
__device__ __forceinline__ void quad_stage(const StageArgs<R>& a) {
  constexpr int NP = NPQ, NFP = NFPQ, NH = QD_NH;
  constexpr int I0 = P * NH;        // first output node of this half
  constexpr int F0 = 2 * P;         // first own face
  constexpr int FX = 2 - 2 * P;     // first face of the other half
  constexpr int VS = 6 * NP * TILE;
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  const int64_t tile = blockIdx.x;
  if (tile * TILE >= a.nti) return;  // whole blocks only
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  const int half = l & 1;  // 0: owns E, computes Phi_H;  1: owns H, computes Phi_E
  const int lane = (w >> 1) * 16 + (l >> 1);
  const int prob = a.tprob ? a.tprob[tile] : 0;
  const StageCoef<R> cf = a.coef[prob];
  if (!cf.active) return;  // tile-uniform
  const int cOwn = half ? 3 : 0, cOut = half ? 0 : 3;
  const R sH = a.sH;
  const R sIn = half ? sH : R(1);
  const R sOut = half ? R(1) : sH;
  const R pec = half ? R(0) : R(-2);

  R G[9];
  const R* gv = a.gvol + tile * GV * TILE + lane;
#pragma unroll
  for (int m = 0; m < 9; ++m) G[m] = gv[m * TILE];
  const R sv = half ? -gv[9 * TILE] : gv[10 * TILE] * sOut;
  int32_t code[2];
  R fn[2][3], fk1[2], fk2[2];
#pragma unroll
  for (int ff = 0; ff < 2; ++ff) {
    const int f = F0 + ff;
    code[ff] = a.nbr[(tile * 4 + f) * TILE + lane];
    const R* gf = a.gface + (tile * 4 + f) * GF * TILE + lane;
    fn[ff][0] = gf[0];
    fn[ff][1] = gf[TILE];
    fn[ff][2] = gf[2 * TILE];
    fk1[ff] = gf[(3 + 2 * half) * TILE] * sOut;
    fk2[ff] = gf[(4 + 2 * half) * TILE] * sOut;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* tr = reinterpret_cast<R*>(smem_raw) + threadIdx.x;  // slot k at tr[k * QD_THREADS]
  R* fx = tr + QD_FSLOTS * QD_THREADS;                    // fluxes handed to the other half
  R* bs = fx + QD_FSLOTS * QD_THREADS;                    // base rows

  grid_dep_wait();
  if (a.pactive && !a.pactive[prob]) return;  // tile-uniform; written by the CG kernels
  R v[3][NP];
  {
    const R* vin = a.vin + tile * VS + cOwn * NP * TILE + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) v[c][n] = sIn * vin[(c * NP + n) * TILE];
  }
  const int64_t off = tile * VS + cOut * NP * TILE + lane;
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) {
        R* dst = bs + (c * NH + ii) * QD_THREADS;
        const R* src = a.base + off + (c * NP + I0 + ii) * TILE;
        if constexpr (sizeof(R) == 4) cp_async_4(dst, src);
        else cp_async_8(dst, src);
      }
  }
#pragma unroll
  for (int ff = 0; ff < 2; ++ff) {
    if (code[ff] >= 0) {
      const int64_t k = int64_t(code[ff] >> 5);
      const R* nb = a.vin + (k >> 5) * VS + cOwn * NP * TILE + (k & 31);
      const int tab = (((code[ff] >> 3) & 3) * 6 + (code[ff] & 7)) * NFP;
#pragma unroll
      for (int jf = 0; jf < NFP; ++jf) {
        const int nn = cNB[tab + jf];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          R* dst = tr + ((ff * NFP + jf) * 3 + c) * QD_THREADS;
          if constexpr (sizeof(R) == 4) cp_async_4(dst, nb + (c * NP + nn) * TILE);
          else cp_async_8(dst, nb + (c * NP + nn) * TILE);
        }
      }
    }
  }
  cp_async_commit();

  R phi[3][NH];
#pragma unroll
  for (int ii = 0; ii < NH; ++ii) {
    const int i = I0 + ii;
    R d[3][3];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < 3; ++c) d[b][c] = R(0);
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      const R dr = cD<R>((0 * NP + i) * NP + j), ds = cD<R>((1 * NP + i) * NP + j), dt = cD<R>((2 * NP + i) * NP + j);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d[0][c] = fma(dr, v[c][j], d[0][c]);
        d[1][c] = fma(ds, v[c][j], d[1][c]);
        d[2][c] = fma(dt, v[c][j], d[2][c]);
      }
    }
    auto dx = [&](int ax, int c) { return G[0 * 3 + ax] * d[0][c] + G[1 * 3 + ax] * d[1][c] + G[2 * 3 + ax] * d[2][c]; };
    phi[0][ii] = sv * (dx(1, 2) - dx(2, 1));
    phi[1][ii] = sv * (dx(2, 0) - dx(0, 2));
    phi[2][ii] = sv * (dx(0, 1) - dx(1, 0));
  }

  cp_async_wait_all();
  // Own faces: fluxes, their lift onto this half's nodes, and the hand-over.
#pragma unroll
  for (int ff = 0; ff < 2; ++ff) {
    const int f = F0 + ff;
    const R n0 = fn[ff][0], n1 = fn[ff][1], n2 = fn[ff][2];
    const R k1 = fk1[ff], k2 = fk2[ff];
    const bool interior = code[ff] >= 0;
    const R bscale = code[ff] == NBR_PEC ? pec : R(-1);
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      const int own = FM.v[f][jf];
      R X[3], Y[3];
      if (interior) {
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = sIn * tr[((ff * NFP + jf) * 3 + c) * QD_THREADS] - v[c][own];
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) X[c] = bscale * v[c][own];
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[c] = __shfl_xor_sync(0xffffffffu, X[c], 1);
      const R nY = n0 * Y[0] + n1 * Y[1] + n2 * Y[2];
      R fl[3];
      fl[0] = k1 * (n1 * X[2] - n2 * X[1]) + k2 * (Y[0] - n0 * nY);
      fl[1] = k1 * (n2 * X[0] - n0 * X[2]) + k2 * (Y[1] - n1 * nY);
      fl[2] = k1 * (n0 * X[1] - n1 * X[0]) + k2 * (Y[2] - n2 * nY);
#pragma unroll
      for (int c = 0; c < 3; ++c) fx[((ff * NFP + jf) * 3 + c) * QD_THREADS] = fl[c];
      if constexpr (P == 0) {  // faces 0, 1 come first in the lift sum
#pragma unroll
        for (int ii = 0; ii < NH; ++ii) {
          const R L = cL<R>((I0 + ii) * 4 * NFP + f * NFP + jf);
#pragma unroll
          for (int c = 0; c < 3; ++c) phi[c][ii] = fma(L, fl[c], phi[c][ii]);
        }
      }
    }
  }
  quad_barrier();
  // Faces 0, 1 then 2, 3, as in dg_stage_kernel: the half owning faces 2, 3 first
  // lifts the other half's faces 0, 1, then its own (read back from its slots).
  const R* fxo = fx - threadIdx.x + (threadIdx.x ^ 32);  // the other half's hand-over slots
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const bool mine = (P == 0) ? false : (g == 1);
    if (P == 0 && g == 0) continue;  // own faces 0, 1 already lifted
    const R* src = mine ? fx : fxo;
    const int fbase = mine ? F0 : FX;
#pragma unroll
    for (int ff = 0; ff < 2; ++ff) {
      const int f = fbase + ff;
#pragma unroll
      for (int jf = 0; jf < NFP; ++jf) {
        R fl[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) fl[c] = src[((ff * NFP + jf) * 3 + c) * QD_THREADS];
#pragma unroll
        for (int ii = 0; ii < NH; ++ii) {
          const R L = cL<R>((I0 + ii) * 4 * NFP + f * NFP + jf);
#pragma unroll
          for (int c = 0; c < 3; ++c) phi[c][ii] = fma(L, fl[c], phi[c][ii]);
        }
      }
    }
  }

  if (half && a.sigma) {  // conductivity: Phi_E -= (sigma / eps) E on this half's nodes
    const R so = a.gvol[(tile * GV + 11) * TILE + lane];
    const R* ev = a.vin + tile * VS + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) phi[c][ii] -= so * ev[(c * NP + I0 + ii) * TILE];
  }
  if (half && a.jre) add_source<R, NH>(phi, a, cf, tile, lane, I0);  // source on the E rows
  if (a.bre) {  // impedance-face data on this thread's output rows
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) {
        const int64_t o = off + (c * NP + I0 + ii) * TILE;
        phi[c][ii] += cf.s_cos * a.bre[o] - cf.s_sin * a.bim[o];
      }
  }
  if (a.fre) accumulate_filter<R, NH>(a, cf, phi, off, I0);
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int ii = 0; ii < NH; ++ii) {
        const int64_t o = off + (c * NP + I0 + ii) * TILE;
        a.out[o] = bs[(c * NH + ii) * QD_THREADS] + cf.c_out * phi[c][ii];
      }
  }
}

template <typename R, int MINB>
__global__ void __launch_bounds__(QD_THREADS, MINB) dg_stage_quad(const StageArgs<R> a) {
  grid_dep_launch();
  if ((threadIdx.x >> 5) & 1) quad_stage<R, 1>(a);
  else quad_stage<R, 0>(a);
}

#include "dg_stage_tc.cuh"

}  // namespace

// Dynamic shared memory of the two-thread kernel: the trace slots, plus the prefetched
// source rows in single-frequency source stages (src = true).
template <typename R>
constexpr size_t stage_smem(bool src = false) {
  return size_t(TRACE_SLOTS + (src ? 3 * NPQ : 0)) * STAGE_THREADS * sizeof(R);
}
template <typename R>
bool prefetches_source(const StageArgs<R>& a) {
  return a.jre != nullptr && a.nharm <= 0;
}

template <typename Arg>
void launch_k(void (*k)(Arg), unsigned blocks, unsigned threads, size_t smem, cudaStream_t s, bool pdl,
              const Arg& a) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, a);
}

template <>
void launch_stage<CMCG_Q, float>(const StageArgs<float>& a, cudaStream_t s, int form, bool pdl) {
  const unsigned blocks = unsigned((2 * a.nti + STAGE_THREADS - 1) / STAGE_THREADS);
  const unsigned qblocks = unsigned(a.nti / TILE);  // one block per tile
  const size_t sm = stage_smem<float>(prefetches_source(a));
  constexpr size_t qsm = quad_smem<float>();
  switch (form) {
    case 1: launch_k(dg_stage_kernel<float, 3>, blocks, STAGE_THREADS, sm, s, pdl, a); break;
    case 2: launch_k(dg_stage_kernel<float, 4>, blocks, STAGE_THREADS, sm, s, pdl, a); break;
    case 3: launch_k(dg_stage_quad<float, 4>, qblocks, QD_THREADS, qsm, s, pdl, a); break;
    case 4: launch_k(dg_stage_quad<float, 5>, qblocks, QD_THREADS, qsm, s, pdl, a); break;
    case 5: launch_k(dg_stage_quad<float, 6>, qblocks, QD_THREADS, qsm, s, pdl, a); break;
    case STAGE_FORM_TC:
      launch_k(dg_stage_tc<TC_MINB>, unsigned((a.nti + TC_TETS - 1) / TC_TETS), TC_THREADS,
               tc_smem(prefetches_source(a)), s, pdl, a);
      break;
    default: launch_k(dg_stage_kernel<float, 1>, blocks, STAGE_THREADS, sm, s, pdl, a); break;
  }
}
template <>
void launch_stage<CMCG_Q, double>(const StageArgs<double>& a, cudaStream_t s, int form, bool pdl) {
  const unsigned blocks = unsigned((2 * a.nti + STAGE_THREADS - 1) / STAGE_THREADS);
  const unsigned qblocks = unsigned(a.nti / TILE);
  constexpr size_t qsm = quad_smem<double>();
  switch (form) {
    case 1: launch_k(dg_stage_quad<double, 2>, qblocks, QD_THREADS, qsm, s, pdl, a); break;
    case 2: launch_k(dg_stage_quad<double, 3>, qblocks, QD_THREADS, qsm, s, pdl, a); break;
    default: launch_k(dg_stage_kernel<double, 1>, blocks, STAGE_THREADS, stage_smem<double>(prefetches_source(a)), s, pdl, a); break;
  }
}

template <>
void upload_constants<CMCG_Q>(const RefMats& rm) {
  // allow the dynamic shared memory of the trace prefetch beyond the 48 KiB default
  cudaFuncSetAttribute(dg_stage_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>(true)));
  cudaFuncSetAttribute(dg_stage_kernel<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>(true)));
  cudaFuncSetAttribute(dg_stage_kernel<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>(true)));
  cudaFuncSetAttribute(dg_stage_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<double>(true)));
  cudaFuncSetAttribute(dg_stage_quad<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(quad_smem<float>()));
  cudaFuncSetAttribute(dg_stage_quad<float, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(quad_smem<float>()));
  cudaFuncSetAttribute(dg_stage_quad<float, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(quad_smem<float>()));
  cudaFuncSetAttribute(dg_stage_quad<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(quad_smem<double>()));
  cudaFuncSetAttribute(dg_stage_quad<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(quad_smem<double>()));
  cudaFuncSetAttribute(dg_stage_tc<TC_MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc_smem(true)));
  cudaFuncSetAttribute(dg_stage_tc<TC_MINB>, cudaFuncAttributePreferredSharedMemoryCarveout,
                       int(cudaSharedmemCarveoutMaxShared));  // two P3 CTAs per SM need 2 x 113 KB
  tc_upload_reference(rm);
  const int np = rm.np, nfp = rm.nfp;
  std::vector<double> D(3 * np * np);
  for (int i = 0; i < np * np; ++i) {
    D[i] = rm.Dr[i];
    D[np * np + i] = rm.Ds[i];
    D[2 * np * np + i] = rm.Dt[i];
  }
  std::vector<float> Df(D.begin(), D.end()), Lf(rm.LIFT.begin(), rm.LIFT.end());
  std::vector<signed char> nbv(rm.nbrnode.begin(), rm.nbrnode.end());
  cudaMemcpyToSymbol(cDd, D.data(), sizeof(double) * D.size());
  cudaMemcpyToSymbol(cDf, Df.data(), sizeof(float) * Df.size());
  cudaMemcpyToSymbol(cLd, rm.LIFT.data(), sizeof(double) * rm.LIFT.size());
  cudaMemcpyToSymbol(cLf, Lf.data(), sizeof(float) * Lf.size());
  cudaMemcpyToSymbol(cNB, nbv.data(), nbv.size());
  (void)nfp;
}

}  // namespace cmcg
