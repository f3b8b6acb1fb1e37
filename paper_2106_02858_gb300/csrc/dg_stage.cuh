// One explicit Runge-Kutta stage of the DG time-domain Maxwell scheme, for a
// fixed polynomial order CMCG_Q (included once per order by dg_q{1,2,3}.cu).
//
// Each thread owns one tetrahedron K and evaluates, for its stage input v,
//
//   Phi_E = -eps^{-1} curl H + LIFT . fE,    Phi_H = mu^{-1} curl E + LIFT . fH
//
// (Eq. ode_system: Phi(t, U) = Re(J e^{i w t}) + B U, strong form of the 3D
// upwind DG operator generalising Eq. DG_semidiscrete), with face terms written
// in jump form dE = E^+ - E^-, dH = H^+ - H^-:
//
//   fE = aE (dE - n (n . dE)) - bE (n x dH)
//   fH = bH (n x dE)          + aH (dH - n (n . dH))
//
//   aE = fscale / (eps (Z^- + Z^+)),  bE = Z^+ aE,  aH = fscale / (mu (Y^- + Y^+)),  bH = Y^+ aH
//
// which is -n x (H^ - H^-) and n x (E^ - E^-) for the upwind traces
// E^ = (Y^- E^- + Y^+ E^+ - (H^- - H^+) x n) / (Y^- + Y^+),
// H^ = (Z^- H^- + Z^+ H^+ + (E^- - E^+) x n) / (Z^- + Z^+); PEC faces use the
// mirror state (dE = -2 E^-, dH = 0), impedance faces the zero state
// (dE = -E^-, dH = -H^-).  fscale = |F| / (|F_ref| |det A|) folds the
// block-diagonal inverse mass (Eq. ode_system) into the lift.  The adjoint
// stage (Section 4.1.2, P* = Sigma P Sigma) flips the sign of every magnetic
// value read and of Phi_H (sH = -1): no extra memory pass.
//
// Reference matrices D_r, D_s, D_t and LIFT live in constant memory; with the
// loops unrolled their indices are compile-time constants, so they are read as
// constant-bank operands of the FMAs.
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

template <typename R>
__global__ void __launch_bounds__(128) dg_stage_kernel(const StageArgs<R> a) {
  constexpr int NP = NPQ, NFP = NFPQ;
  constexpr int VS = 6 * NP * TILE;  // elements per tile of a field vector
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (gt >= a.nti) return;
  const int64_t tile = gt >> 5;
  const int lane = int(gt & 31);
  const R sH = a.sH;

  R u[6][NP];
  {
    const R* vin = a.vin + tile * VS + lane;
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) u[c][n] = vin[(c * NP + n) * TILE];
#pragma unroll
    for (int c = 3; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) u[c][n] *= sH;
  }

  R phi[6][NP];
  {
    const R* gv = a.gvol + tile * GV * TILE + lane;
    R G[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) G[m] = gv[m * TILE];
    const R ie = gv[9 * TILE], im = gv[10 * TILE];
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      R d[3][6];
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int c = 0; c < 6; ++c) d[b][c] = R(0);
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        const R dr = cD<R>((0 * NP + i) * NP + j), ds = cD<R>((1 * NP + i) * NP + j), dt = cD<R>((2 * NP + i) * NP + j);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          d[0][c] = fma(dr, u[c][j], d[0][c]);
          d[1][c] = fma(ds, u[c][j], d[1][c]);
          d[2][c] = fma(dt, u[c][j], d[2][c]);
        }
      }
      // d/dx_ax of component c = sum_b G[b][ax] d[b][c]
      auto dx = [&](int ax, int c) { return G[0 * 3 + ax] * d[0][c] + G[1 * 3 + ax] * d[1][c] + G[2 * 3 + ax] * d[2][c]; };
      phi[0][i] = -ie * (dx(1, 5) - dx(2, 4));
      phi[1][i] = -ie * (dx(2, 3) - dx(0, 5));
      phi[2][i] = -ie * (dx(0, 4) - dx(1, 3));
      phi[3][i] = im * (dx(1, 2) - dx(2, 1));
      phi[4][i] = im * (dx(2, 0) - dx(0, 2));
      phi[5][i] = im * (dx(0, 1) - dx(1, 0));
    }
  }

#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const R* gf = a.gface + (tile * 4 + f) * GF * TILE + lane;
    const R n0 = gf[0], n1 = gf[TILE], n2 = gf[2 * TILE];
    const R aE = gf[3 * TILE], bE = gf[4 * TILE], aH = gf[5 * TILE], bH = gf[6 * TILE];
    const int32_t code = a.nbr[(tile * 4 + f) * TILE + lane];
    const R* nb = a.vin;
    int tab = 0;
    if (code >= 0) {
      const int64_t k = int64_t(code >> 5);
      nb = a.vin + (k >> 5) * VS + (k & 31);
      tab = (((code >> 3) & 3) * 6 + (code & 7)) * NFP;
    }
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      const int own = FM.v[f][jf];
      R dE[3], dH[3];
      if (code >= 0) {
        const int nn = cNB[tab + jf];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dE[c] = nb[(c * NP + nn) * TILE] - u[c][own];
          dH[c] = sH * nb[((3 + c) * NP + nn) * TILE] - u[3 + c][own];
        }
      } else if (code == NBR_PEC) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dE[c] = R(-2) * u[c][own];
          dH[c] = R(0);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          dE[c] = -u[c][own];
          dH[c] = -u[3 + c][own];
        }
      }
      const R ndE = n0 * dE[0] + n1 * dE[1] + n2 * dE[2];
      const R ndH = n0 * dH[0] + n1 * dH[1] + n2 * dH[2];
      const R xE0 = n1 * dE[2] - n2 * dE[1], xE1 = n2 * dE[0] - n0 * dE[2], xE2 = n0 * dE[1] - n1 * dE[0];
      const R xH0 = n1 * dH[2] - n2 * dH[1], xH1 = n2 * dH[0] - n0 * dH[2], xH2 = n0 * dH[1] - n1 * dH[0];
      R fE[3], fH[3];
      fE[0] = aE * (dE[0] - n0 * ndE) - bE * xH0;
      fE[1] = aE * (dE[1] - n1 * ndE) - bE * xH1;
      fE[2] = aE * (dE[2] - n2 * ndE) - bE * xH2;
      fH[0] = bH * xE0 + aH * (dH[0] - n0 * ndH);
      fH[1] = bH * xE1 + aH * (dH[1] - n1 * ndH);
      fH[2] = bH * xE2 + aH * (dH[2] - n2 * ndH);
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        const R L = cL<R>(i * 4 * NFP + f * NFP + jf);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          phi[c][i] = fma(L, fE[c], phi[c][i]);
          phi[3 + c][i] = fma(L, fH[c], phi[3 + c][i]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 3; c < 6; ++c)
#pragma unroll
    for (int n = 0; n < NP; ++n) phi[c][n] *= sH;

  const int64_t off = tile * VS + lane;
  if (a.jre) {
    const int64_t joff = tile * (3 * NP * TILE) + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = joff + (c * NP + n) * TILE;
        phi[c][n] += a.s_cos * a.jre[o] - a.s_sin * a.jim[o];
      }
  }
  if (a.fre) {  // forward sweeps only (u holds the unflipped stage input)
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        a.fre[o] += a.fa_re * u[c][n] + a.fb_re * phi[c][n];
        a.fim[o] += a.fa_im * u[c][n] + a.fb_im * phi[c][n];
      }
  }
  if (a.acc_out) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        a.acc_out[o] = a.acc_in[o] + a.c_acc * phi[c][n];
      }
  }
  if (a.out) {
#pragma unroll
    for (int c = 0; c < 6; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) {
        const int64_t o = off + (c * NP + n) * TILE;
        a.out[o] = a.base[o] + a.c_out * phi[c][n];
      }
  }
}

}  // namespace

template <>
void launch_stage<CMCG_Q, float>(const StageArgs<float>& a, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (a.nti + threads - 1) / threads;
  dg_stage_kernel<float><<<(unsigned)blocks, threads, 0, s>>>(a);
}
template <>
void launch_stage<CMCG_Q, double>(const StageArgs<double>& a, cudaStream_t s) {
  const int threads = 128;
  const int64_t blocks = (a.nti + threads - 1) / threads;
  dg_stage_kernel<double><<<(unsigned)blocks, threads, 0, s>>>(a);
}

template <>
void upload_constants<CMCG_Q>(const RefMats& rm) {
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
