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
__constant__ float2 cD2[3 * NPQ * NPQ];      // (D, D) pairs for the packed kernel
__constant__ float2 cL2[NPQ * 4 * NFPQ];     // (LIFT, LIFT) pairs

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
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// MINB: minimum resident blocks per SM requested from the compiler (caps registers at
// 65536 / (MINB * STAGE_THREADS)); the forms are timed per handle (see api.cu).
template <typename R, int MINB>
__global__ void __launch_bounds__(STAGE_THREADS, MINB) dg_stage_kernel(const StageArgs<R> a) {
  constexpr int NP = NPQ, NFP = NFPQ;
  constexpr int VS = 6 * NP * TILE;  // elements per tile of a field vector
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  const int64_t gthr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gt = gthr >> 1;  // tetrahedron; nti is a multiple of 32, so whole warps leave together
  if (gt >= a.nti) return;
  const int half = int(gthr & 1);  // 0: owns E, computes Phi_H;  1: owns H, computes Phi_E
  const int64_t tile = gt >> 5;
  const int lane = int(gt & 31);
  // A warp (16 tetrahedra) lies inside one tile, hence inside one problem: uniform exits.
  const int prob = a.tprob ? a.tprob[tile] : 0;
  if (a.pactive && !a.pactive[prob]) return;
  const StageCoef<R> cf = a.coef[prob];
  if (!cf.active) return;
  const int cOwn = half ? 3 : 0, cOut = half ? 0 : 3;
  const R sH = a.sH;
  const R sIn = half ? sH : R(1);   // sign of the own field (magnetic values flipped in the adjoint)
  const R sOut = half ? R(1) : sH;  // sign of Phi_H
  const R pec = half ? R(0) : R(-2);  // PEC mirror: dE = -2 E^-, dH = 0

  R v[3][NP];
  {
    const R* vin = a.vin + tile * VS + cOwn * NP * TILE + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) v[c][n] = sIn * vin[(c * NP + n) * TILE];
  }

  // Independent loads first (affine factors, codes, face coefficients, base rows),
  // then the neighbour traces into shared memory (their addresses need the codes).
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
      R fl[3];
      fl[0] = k1 * (n1 * X[2] - n2 * X[1]) + k2 * (Y[0] - n0 * nY);
      fl[1] = k1 * (n2 * X[0] - n0 * X[2]) + k2 * (Y[1] - n1 * nY);
      fl[2] = k1 * (n0 * X[1] - n1 * X[0]) + k2 * (Y[2] - n2 * nY);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const R L = cL<R>(i * 4 * NFP + f * NFP + jf);
#pragma unroll
        for (int c = 0; c < 3; ++c) phi[c][i] = fma(L, fl[c], phi[c][i]);
      }
    }
  }

  if (half && a.jre) {  // source on the E rows
    const int64_t joff = tile * (3 * NP * TILE) + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = joff + (c * NP + n) * TILE;
        phi[c][n] += cf.s_cos * a.jre[o] - cf.s_sin * a.jim[o];
      }
  }
  if (a.fre) {  // forward sweeps only: F += fa U + fb Phi on this thread's output rows
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        const R u = a.vin[o];
        a.fre[o] += cf.fa_re * u + cf.fb_re * phi[c][n];
        a.fim[o] += cf.fa_im * u + cf.fb_im * phi[c][n];
      }
  }
  if (a.acc_out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        a.acc_out[o] = a.acc_in[o] + cf.c_acc * phi[c][n];
      }
  }
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

// Packed FP32 stage (sm_100+ f32x2 FMA): each lane handles two adjacent
// tetrahedra (2k, 2k + 1 of its 32-tet tile) in one role (E or H, as above),
// so every per-tetrahedron quantity is a float2 and every FMA a packed FMA with
// the reference-matrix entry duplicated in both halves.  A warp is one tile.
// Neighbour traces are prefetched with cp.async as in the scalar kernel;
// boundary faces zero-fill their slots, and the jump is formed without a
// branch as X = a_nb * trace + a_own * own (a_nb = sign, a_own = -1 on interior
// faces; a_nb = 0, a_own = -2 / 0 / -1 on PEC E / PEC H / impedance faces).
constexpr int PK_THREADS = 128;
constexpr int PK_SLOTS = 4 * NFPQ * 3;  // float2 slots per thread

__device__ __forceinline__ void cp_async_4z(void* smem, const void* gmem, bool fill) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  const int n = fill ? 4 : 0;  // 0: write zeros, read nothing
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

template <int MINB>
__global__ void __launch_bounds__(PK_THREADS, MINB) dg_stage_packed(const StageArgs<float> a) {
  constexpr int NP = NPQ, NFP = NFPQ;
  constexpr int VS = 6 * NP * TILE;
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  const int64_t tile = (int64_t(blockIdx.x) * PK_THREADS + threadIdx.x) >> 5;
  if (tile * TILE >= a.nti) return;
  const int prob = a.tprob ? a.tprob[tile] : 0;
  if (a.pactive && !a.pactive[prob]) return;
  const StageCoef<float> cf = a.coef[prob];
  if (!cf.active) return;
  const int lane = threadIdx.x & 31;
  const int half = lane & 1;
  const int t0 = (lane >> 1) * 2;  // first of the lane's two tetrahedra within the tile
  const int cOwn = half ? 3 : 0, cOut = half ? 0 : 3;
  const float sH = a.sH;
  const float sIn = half ? sH : 1.f, sOut = half ? 1.f : sH, pec = half ? 0.f : -2.f;
  const float2 sIn2 = f2(sIn);

  float2 v[3][NP];
  {
    const float* vin = a.vin + tile * VS + cOwn * NP * TILE + t0;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) v[c][n] = mul2(sIn2, *reinterpret_cast<const float2*>(vin + (c * NP + n) * TILE));
  }

  float2 G[9];
  const float* gv = a.gvol + tile * GV * TILE + t0;
#pragma unroll
  for (int m = 0; m < 9; ++m) G[m] = *reinterpret_cast<const float2*>(gv + m * TILE);
  const float2 sv = half ? neg2(*reinterpret_cast<const float2*>(gv + 9 * TILE))
                         : mul2(f2(sOut), *reinterpret_cast<const float2*>(gv + 10 * TILE));
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tr = reinterpret_cast<float2*>(smem_raw) + threadIdx.x;  // slot k at tr[k * PK_THREADS]
  int2 code[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) code[f] = *reinterpret_cast<const int2*>(a.nbr + (tile * 4 + f) * TILE + t0);
  float2 fn[4][3], fk1[4], fk2[4];
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float* gf = a.gface + (tile * 4 + f) * GF * TILE + t0;
#pragma unroll
    for (int m = 0; m < 3; ++m) fn[f][m] = *reinterpret_cast<const float2*>(gf + m * TILE);
    fk1[f] = mul2(f2(sOut), *reinterpret_cast<const float2*>(gf + (3 + 2 * half) * TILE));
    fk2[f] = mul2(f2(sOut), *reinterpret_cast<const float2*>(gf + (4 + 2 * half) * TILE));
  }
  const int64_t off = tile * VS + cOut * NP * TILE + t0;
  float2 bv[3][NP];
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) bv[c][n] = *reinterpret_cast<const float2*>(a.base + off + (c * NP + n) * TILE);
  }
#pragma unroll
  for (int f = 0; f < 4; ++f) {
#pragma unroll
    for (int w = 0; w < 2; ++w) {
      const int32_t cd = w ? code[f].y : code[f].x;
      const bool in = cd >= 0;
      const int64_t k = in ? int64_t(cd >> 5) : 0;
      const float* nb = a.vin + (k >> 5) * VS + cOwn * NP * TILE + (k & 31);
      const int tab = in ? (((cd >> 3) & 3) * 6 + (cd & 7)) * NFP : 0;
#pragma unroll
      for (int jf = 0; jf < NFP; ++jf) {
        const int nn = in ? int(cNB[tab + jf]) : 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          cp_async_4z(reinterpret_cast<float*>(tr + ((f * NFP + jf) * 3 + c) * PK_THREADS) + w,
                      nb + (c * NP + nn) * TILE, in);
      }
    }
  }
  cp_async_commit();

  float2 phi[3][NP];
  {
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      float2 d[3][3];
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 3; ++c) d[b][c] = f2(0.f);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const float2 dr = cD2[(0 * NP + i) * NP + j], ds = cD2[(1 * NP + i) * NP + j], dt = cD2[(2 * NP + i) * NP + j];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          d[0][c] = fma2(dr, v[c][j], d[0][c]);
          d[1][c] = fma2(ds, v[c][j], d[1][c]);
          d[2][c] = fma2(dt, v[c][j], d[2][c]);
        }
      }
      auto dx = [&](int ax, int c) {
        return fma2(G[2 * 3 + ax], d[2][c], fma2(G[1 * 3 + ax], d[1][c], mul2(G[0 * 3 + ax], d[0][c])));
      };
      phi[0][i] = mul2(sv, add2(dx(1, 2), neg2(dx(2, 1))));
      phi[1][i] = mul2(sv, add2(dx(2, 0), neg2(dx(0, 2))));
      phi[2][i] = mul2(sv, add2(dx(0, 1), neg2(dx(1, 0))));
    }
  }

  cp_async_wait_all();
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const float2 n0 = fn[f][0], n1 = fn[f][1], n2 = fn[f][2];
    const float2 k1 = fk1[f], k2 = fk2[f];
    // jump coefficients per tetrahedron of the pair
    auto anb = [&](int32_t cd) { return cd >= 0 ? sIn : 0.f; };
    auto aown = [&](int32_t cd) { return cd >= 0 ? -1.f : (cd == NBR_PEC ? pec : -1.f); };
    const float2 An = make_float2(anb(code[f].x), anb(code[f].y));
    const float2 Ao = make_float2(aown(code[f].x), aown(code[f].y));
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      const int own = FM.v[f][jf];
      float2 X[3], Y[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) X[c] = fma2(An, tr[((f * NFP + jf) * 3 + c) * PK_THREADS], mul2(Ao, v[c][own]));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        Y[c].x = __shfl_xor_sync(0xffffffffu, X[c].x, 1);
        Y[c].y = __shfl_xor_sync(0xffffffffu, X[c].y, 1);
      }
      const float2 nY = fma2(n2, Y[2], fma2(n1, Y[1], mul2(n0, Y[0])));
      float2 fl[3];
      fl[0] = fma2(k2, fma2(neg2(n0), nY, Y[0]), mul2(k1, fma2(n1, X[2], neg2(mul2(n2, X[1])))));
      fl[1] = fma2(k2, fma2(neg2(n1), nY, Y[1]), mul2(k1, fma2(n2, X[0], neg2(mul2(n0, X[2])))));
      fl[2] = fma2(k2, fma2(neg2(n2), nY, Y[2]), mul2(k1, fma2(n0, X[1], neg2(mul2(n1, X[0])))));
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const float2 L = cL2[i * 4 * NFP + f * NFP + jf];
#pragma unroll
        for (int c = 0; c < 3; ++c) phi[c][i] = fma2(L, fl[c], phi[c][i]);
      }
    }
  }

  if (half && a.jre) {
    const int64_t joff = tile * (3 * NP * TILE) + t0;
    const float2 sc = f2(cf.s_cos), ss = f2(-cf.s_sin);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = joff + (c * NP + n) * TILE;
        phi[c][n] = fma2(sc, *reinterpret_cast<const float2*>(a.jre + o),
                         fma2(ss, *reinterpret_cast<const float2*>(a.jim + o), phi[c][n]));
      }
  }
  if (a.fre) {
    const float2 far = f2(cf.fa_re), fai = f2(cf.fa_im), fbr = f2(cf.fb_re), fbi = f2(cf.fb_im);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        const float2 u = *reinterpret_cast<const float2*>(a.vin + o);
        float2* Fr = reinterpret_cast<float2*>(a.fre + o);
        float2* Fi = reinterpret_cast<float2*>(a.fim + o);
        *Fr = fma2(far, u, fma2(fbr, phi[c][n], *Fr));
        *Fi = fma2(fai, u, fma2(fbi, phi[c][n], *Fi));
      }
  }
  if (a.acc_out) {
    const float2 ca = f2(cf.c_acc);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        *reinterpret_cast<float2*>(a.acc_out + o) = fma2(ca, phi[c][n], *reinterpret_cast<const float2*>(a.acc_in + o));
      }
  }
  if (a.out) {
    const float2 co = f2(cf.c_out);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        *reinterpret_cast<float2*>(a.out + o) = fma2(co, phi[c][n], bv[c][n]);
      }
  }
}

}  // namespace

template <typename R>
constexpr size_t stage_smem() {
  return size_t(TRACE_SLOTS) * STAGE_THREADS * sizeof(R);
}

template <>
void launch_stage<CMCG_Q, float>(const StageArgs<float>& a, cudaStream_t s, int variant) {
  const unsigned blocks = unsigned((2 * a.nti + STAGE_THREADS - 1) / STAGE_THREADS);
  constexpr size_t sm = stage_smem<float>();
  switch (variant) {
    case 1: dg_stage_kernel<float, 3><<<blocks, STAGE_THREADS, sm, s>>>(a); break;
    case 2: dg_stage_kernel<float, 4><<<blocks, STAGE_THREADS, sm, s>>>(a); break;
    default: dg_stage_kernel<float, 1><<<blocks, STAGE_THREADS, sm, s>>>(a); break;
  }
}
template <>
void launch_stage<CMCG_Q, double>(const StageArgs<double>& a, cudaStream_t s, int) {
  const unsigned blocks = unsigned((2 * a.nti + STAGE_THREADS - 1) / STAGE_THREADS);
  dg_stage_kernel<double, 1><<<blocks, STAGE_THREADS, stage_smem<double>(), s>>>(a);
}

template <>
void launch_stage_packed<CMCG_Q>(const StageArgs<float>& a, cudaStream_t s, int minb) {
  const unsigned blocks = unsigned((a.nti + PK_THREADS - 1) / PK_THREADS);  // one warp per 32-tet tile
  const size_t sm = size_t(PK_SLOTS) * PK_THREADS * sizeof(float2);
  (void)minb;
  dg_stage_packed<2><<<blocks, PK_THREADS, sm, s>>>(a);
}

template <>
void upload_constants<CMCG_Q>(const RefMats& rm) {
  {
    const int sm = int(size_t(PK_SLOTS) * PK_THREADS * sizeof(float2));
    cudaFuncSetAttribute((const void*)dg_stage_packed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  }
  // allow the dynamic shared memory of the trace prefetch beyond the 48 KiB default
  cudaFuncSetAttribute(dg_stage_kernel<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>()));
  cudaFuncSetAttribute(dg_stage_kernel<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>()));
  cudaFuncSetAttribute(dg_stage_kernel<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<float>()));
  cudaFuncSetAttribute(dg_stage_kernel<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(stage_smem<double>()));
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
  std::vector<float2> D2(D.size()), L2(rm.LIFT.size());
  for (size_t i = 0; i < D.size(); ++i) D2[i] = make_float2(float(D[i]), float(D[i]));
  for (size_t i = 0; i < rm.LIFT.size(); ++i) L2[i] = make_float2(float(rm.LIFT[i]), float(rm.LIFT[i]));
  cudaMemcpyToSymbol(cD2, D2.data(), sizeof(float2) * D2.size());
  cudaMemcpyToSymbol(cL2, L2.data(), sizeof(float2) * L2.size());
  (void)nfp;
}

}  // namespace cmcg
