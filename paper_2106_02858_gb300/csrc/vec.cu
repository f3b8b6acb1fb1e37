// Vector kernels of the CMCG outer loop (Section 2.2, Algorithm cmcg):
// layout conversion between the boundary layout [tet][comp][node] (double) and
// the device layout [tile][comp][node][lane], fused CG updates, and the
// (eps, mu)-weighted inner product (Eq. innerproduct)
//     (X, Y) = sum_K |det A_K| sum_c w_c sum_ij X_c[i] Mref[i][j] Y_c[j],
// w_c = eps_K on E rows, mu_K on H rows, accumulated in FP64 whatever the
// storage precision.  Reductions are deterministic: one partial per block
// (warp shuffles, then shared memory in a fixed order) and one finalising
// block that sums the partials in a fixed order.
#include "common.h"

namespace cmcg {
namespace {


__constant__ double cM1[4 * 4];
__constant__ double cM2[10 * 10];
__constant__ double cM3[20 * 20];

template <int Q>
__device__ __forceinline__ double cM(int idx) {
  if constexpr (Q == 1) return cM1[idx];
  else if constexpr (Q == 2) return cM2[idx];
  else return cM3[idx];
}

template <typename R>
__global__ void to_internal_kernel(const double* __restrict__ ext, int ncomp_ext, int c_ext0, R* __restrict__ in,
                                   int ncomp_in, int c_in0, int cnt, const int32_t* __restrict__ e_of_i, int64_t nti,
                                   int np, double scale, const double* __restrict__ per_tet) {
  const int64_t total = nti * cnt * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int lane = int(idx % TILE);
    const int64_t r = idx / TILE;
    const int n = int(r % np);
    const int c = int((r / np) % cnt);
    const int64_t tile = r / ((int64_t)np * cnt);
    const int32_t e = e_of_i[tile * TILE + lane];
    R v = R(0);
    if (e >= 0) {
      double x = ext[((int64_t)e * ncomp_ext + c_ext0 + c) * np + n] * scale;
      if (per_tet) x *= per_tet[e];
      v = R(x);
    }
    in[((tile * ncomp_in + c_in0 + c) * np + n) * TILE + lane] = v;
  }
}

template <typename R>
__global__ void to_external_kernel(const R* __restrict__ in, int ncomp_in, int c_in0, double* __restrict__ ext,
                                   int ncomp_ext, int c_ext0, int cnt, const int32_t* __restrict__ e_of_i, int64_t nti,
                                   int np) {
  const int64_t total = nti * cnt * np;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int lane = int(idx % TILE);
    const int64_t r = idx / TILE;
    const int n = int(r % np);
    const int c = int((r / np) % cnt);
    const int64_t tile = r / ((int64_t)np * cnt);
    const int32_t e = e_of_i[tile * TILE + lane];
    if (e >= 0) ext[((int64_t)e * ncomp_ext + c_ext0 + c) * np + n] = double(in[((tile * ncomp_in + c_in0 + c) * np + n) * TILE + lane]);
  }
}

// o = a x + b y on the tiles of the problems with mask[p] != 0 (problem of tile t: tprob[t], or 0).
template <typename R>
__global__ void lincomb_masked_kernel(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n,
                                      int64_t tile_len, const int32_t* tprob, const int32_t* mask) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = tprob ? tprob[i / tile_len] : 0;
    if (!mask[p]) continue;
    double v = a * double(x[i]);
    if (y) v += b * double(y[i]);
    const R r = R(v);
    if (o1) o1[i] = r;
    if (o2) o2[i] = r;
    if (o3) o3[i] = r;
  }
}

template <typename R>
__global__ void lincomb_kernel(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = a * double(x[i]);
    if (y) v += b * double(y[i]);
    const R r = R(v);
    if (o1) o1[i] = r;
    if (o2) o2[i] = r;
    if (o3) o3[i] = r;
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[DOT_THREADS / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();  // a previous call's reads of sh are done
  if (l == 0) sh[w] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < DOT_THREADS / 32; ++i) s += sh[i];
  return s;
}

// Per-tet weighted dot of X and Y (vectors in device layout).
template <int Q, typename R>
__device__ __forceinline__ double tet_dot(const R* X, const R* Y, int64_t tile, int lane, const double* wdot) {
  constexpr int NP = np_of(Q);
  const R* x = X + tile * (6 * NP * TILE) + lane;
  const R* y = Y + tile * (6 * NP * TILE) + lane;
  const double wE = wdot[(tile * 2 + 0) * TILE + lane], wH = wdot[(tile * 2 + 1) * TILE + lane];
  double total = 0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double yv[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) yv[j] = double(y[(c * NP + j) * TILE]);
    double s = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double t = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) t = fma(cM<Q>(i * NP + j), yv[j], t);
      s = fma(double(x[(c * NP + i) * TILE]), t, s);
    }
    total += (c < 3 ? wE : wH) * s;
  }
  return total;
}

// (X, Y) and (X, X) of one tetrahedron in one pass over X (each sum in the order of tet_dot).
template <int Q, typename R>
__device__ __forceinline__ void tet_dot2(const R* X, const R* Y, int64_t tile, int lane, const double* wdot,
                                         double& xy, double& xx) {
  constexpr int NP = np_of(Q);
  const R* x = X + tile * (6 * NP * TILE) + lane;
  const R* y = Y + tile * (6 * NP * TILE) + lane;
  const double wE = wdot[(tile * 2 + 0) * TILE + lane], wH = wdot[(tile * 2 + 1) * TILE + lane];
  xy = 0;
  xx = 0;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    double xv[NP], yv[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
      xv[j] = double(x[(c * NP + j) * TILE]);
      yv[j] = double(y[(c * NP + j) * TILE]);
    }
    double s = 0, s2 = 0;
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      double t = 0, t2 = 0;
#pragma unroll
      for (int j = 0; j < NP; ++j) {
        t = fma(cM<Q>(i * NP + j), yv[j], t);
        t2 = fma(cM<Q>(i * NP + j), xv[j], t2);
      }
      s = fma(xv[i], t, s);
      s2 = fma(xv[i], t2, s2);
    }
    xy += (c < 3 ? wE : wH) * s;
    xx += (c < 3 ? wE : wH) * s2;
  }
}

// Block b of the table: its tets, or -1 when past the block's range.
__device__ __forceinline__ int64_t block_tet(const BlockTable& bt) {
  const int b = blockIdx.x;
  return threadIdx.x < bt.ntet[b] ? bt.tet0[b] + threadIdx.x : -1;
}

// A = Uw - WT; partial (D, A).
template <int Q, typename R>
__global__ void __launch_bounds__(DOT_THREADS) cg_after_adjoint_kernel(const R* Uw, const R* WT, R* A, const R* D,
                                                                      const double* wdot, double* partials,
                                                                      const BlockTable bt, const int32_t* pactive) {
  constexpr int NP = np_of(Q);
  const bool act = !pactive || pactive[bt.prob[blockIdx.x]];
  const int64_t t = block_tet(bt);
  double acc = 0, dd = 0;
  if (act && t >= 0) {
    const int64_t tile = t >> 5;
    const int lane = int(t & 31);
    const int64_t base = tile * (6 * NP * TILE) + lane;
#pragma unroll
    for (int k = 0; k < 6 * NP; ++k) A[base + k * TILE] = R(double(Uw[base + k * TILE]) - double(WT[base + k * TILE]));
    tet_dot2<Q, R>(D, A, tile, lane, wdot, acc, dd);
  }
  const double s = block_sum(acc);
  const double s2 = block_sum(dd);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s;
    partials[gridDim.x + blockIdx.x] = s2;
  }
}

// U0 += alpha_p D; R -= alpha_p A; partial (R, R).
template <int Q, typename R>
__global__ void __launch_bounds__(DOT_THREADS) cg_update_kernel(R* U0, R* Rv, const R* D, const R* A, const double* wdot,
                                                               const Scalars* sc, double* partials, const BlockTable bt,
                                                               const int32_t* pactive) {
  constexpr int NP = np_of(Q);
  const int p = bt.prob[blockIdx.x];
  const bool act = !pactive || pactive[p];
  const int64_t t = block_tet(bt);
  double acc = 0;
  if (act && t >= 0) {
    const double alpha = sc[p].alpha;
    const int64_t tile = t >> 5;
    const int lane = int(t & 31);
    const int64_t base = tile * (6 * NP * TILE) + lane;
#pragma unroll
    for (int k = 0; k < 6 * NP; ++k) {
      const int64_t o = base + k * TILE;
      U0[o] = R(double(U0[o]) + alpha * double(D[o]));
      Rv[o] = R(double(Rv[o]) - alpha * double(A[o]));
    }
    acc = tet_dot<Q, R>(Rv, Rv, tile, lane, wdot);
  }
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <int Q, typename R>
__global__ void __launch_bounds__(DOT_THREADS) dot_kernel(const R* X, const R* Y, const double* wdot, double* partials,
                                                         const BlockTable bt) {
  const int64_t t = block_tet(bt);
  const double acc = t >= 0 ? tet_dot<Q, R>(X, Y, t >> 5, int(t & 31), wdot) : 0.0;
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <typename R>
__global__ void scatter_rows_kernel(R* dst_re, R* dst_im, const double* src_re, const double* src_im,
                                    const int64_t* tet, int64_t count, int rows) {
  const int64_t n = count * rows;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / rows, k = i % rows, t = tet[e];
    const int64_t o = (t >> 5) * rows * TILE + k * TILE + (t & 31);
    dst_re[o] = R(src_re[i]);
    dst_im[o] = R(src_im[i]);
  }
}

template <typename R>
__global__ void halo_kernel(R* v, const int64_t* dst, const int64_t* src, int64_t n, int rows) {
  const int64_t total = n * rows;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i / rows, k = i % rows, d = dst[e], s = src[e];
    v[(d >> 5) * rows * TILE + k * TILE + (d & 31)] = v[(s >> 5) * rows * TILE + k * TILE + (s & 31)];
  }
}

__global__ void zero_wdot_kernel(double* wdot, const int64_t* tets, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = tets[i];
    wdot[((t >> 5) * 2 + 0) * TILE + (t & 31)] = 0.0;
    wdot[((t >> 5) * 2 + 1) * TILE + (t & 31)] = 0.0;
  }
}

// gvol item `item` of internal tetrahedra [0, nti) of one problem: val[e] * scale[e] for the
// external tetrahedron e = e_of_i[i] (0 on padding).
template <typename R>
__global__ void set_gvol_item_kernel(R* gvol, int item, const double* val, const double* scale,
                                     const int32_t* e_of_i, int64_t nti) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nti; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = e_of_i[i];
    gvol[((i >> 5) * GV + item) * TILE + (i & 31)] = e >= 0 ? R(val[e] * scale[e]) : R(0);
  }
}

// D = R + beta_p D; Uw = D (active problems only).
template <typename R>
__global__ void cg_direction_kernel(R* D, R* Uw, const R* Rv, const Scalars* sc, const int32_t* tprob,
                                    const int32_t* pactive, int64_t n, int64_t tile_len) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int p = tprob ? tprob[i / tile_len] : 0;
    if (pactive && !pactive[p]) continue;
    const R v = R(double(Rv[i]) + sc[p].beta * double(D[i]));
    D[i] = v;
    Uw[i] = v;
  }
}

__global__ void finalize_kernel(const double* partials, const BlockTable bt, Scalars* sc, int32_t* pactive,
                                const int32_t* used, int which, double tol) {
  __shared__ double sh[256];
  const int p = blockIdx.x;
  const int b0 = bt.coupled ? 0 : bt.pb0[p], b1 = bt.coupled ? bt.nblk : bt.pb0[p + 1];
  auto reduce = [&](const double* part) {
    double s = 0;
    for (int i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
  };
  const double tot = reduce(partials);
  // which == 1: (D, D)_M of the same blocks, stored after the (D, A) partials
  const double dd = which == 1 ? reduce(partials + bt.nblk) : 0.0;
  if (threadIdx.x != 0) return;
  Scalars& S = sc[p];
  if (which == 3) {
    S.rr_new = tot;
    return;
  }
  if (which == 4) {  // as 0, for the problems of `used` only (the others are left untouched)
    if (!used || !used[p]) return;
    S.rr = tot;
    S.rr0 = tot;
    S.iters = 0;
    S.status = isfinite(tot) ? 0 : CMCG_ERR_NONFINITE;
    if (pactive) pactive[p] = (S.status == 0 && tot > 0 && sqrt(tot) > tol * sqrt(tot)) ? 1 : 0;
    return;
  }
  if (which == 0) {
    S.rr = tot;
    S.rr0 = tot;
    S.iters = 0;
    S.status = isfinite(tot) ? 0 : CMCG_ERR_NONFINITE;
    const bool in = !used || used[p];
    if (pactive) pactive[p] = (in && S.status == 0 && tot > 0 && sqrt(tot) > tol * sqrt(tot)) ? 1 : 0;
    return;
  }
  if (pactive && !pactive[p]) return;
  if (!isfinite(tot)) {
    S.status = CMCG_ERR_NONFINITE;
    if (pactive) pactive[p] = 0;
    return;
  }
  if (which == 1) {
    S.dA = tot;
    // (D, A) = |(I - P) D|^2 <= (1 + |P|)^2 |D|^2.  A CFL-stable period map is not a
    // contraction in this norm (non-normal transient growth; |P D| / |D| reaches about 3
    // along the CG directions of the test meshes), but a step beyond the stability limit
    // grows by orders of magnitude per period: |(I - P) D| > 100 |D| means |P| > 99.
    if (tot > 1e4 * dd) {
      S.status = CMCG_ERR_UNSTABLE;
      S.alpha = 0;
      if (pactive) pactive[p] = 0;
    } else if (!(tot > 0)) {
      S.status = CMCG_ERR_CG_BREAKDOWN;
      S.alpha = 0;
      if (pactive) pactive[p] = 0;
    } else {
      S.alpha = S.rr / tot;
    }
  } else {  // which == 2
    S.rr_new = tot;
    S.beta = S.rr > 0 ? tot / S.rr : 0.0;
    S.rr = tot;
    S.iters += 1;
    if (pactive && !(sqrt(tot) > tol * sqrt(S.rr0))) pactive[p] = 0;
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b > 152 * 64) b = 152 * 64;
  if (b < 1) b = 1;
  return int(b);
}

}  // namespace

void upload_dot_mass(int q, const double* M) {
  const int np = np_of(q);
  if (q == 1) cudaMemcpyToSymbol(cM1, M, sizeof(double) * np * np);
  else if (q == 2) cudaMemcpyToSymbol(cM2, M, sizeof(double) * np * np);
  else cudaMemcpyToSymbol(cM3, M, sizeof(double) * np * np);
}

template <typename R>
void launch_to_internal(const double* ext, int ncomp_ext, int c_ext0, R* in, int ncomp_in, int c_in0, int cnt,
                        const int32_t* e_of_i, int64_t nti, int np, double scale, const double* per_tet, cudaStream_t s) {
  const int64_t n = nti * cnt * np;
  to_internal_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(ext, ncomp_ext, c_ext0, in, ncomp_in, c_in0, cnt, e_of_i, nti,
                                                         np, scale, per_tet);
}
template <typename R>
void launch_to_external(const R* in, int ncomp_in, int c_in0, double* ext, int ncomp_ext, int c_ext0, int cnt,
                        const int32_t* e_of_i, int64_t nti, int np, cudaStream_t s) {
  const int64_t n = nti * cnt * np;
  to_external_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(in, ncomp_in, c_in0, ext, ncomp_ext, c_ext0, cnt, e_of_i, nti,
                                                         np);
}
template <typename R>
void launch_lincomb3_masked(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n, int np,
                            const int32_t* tprob, const int32_t* mask, cudaStream_t s) {
  lincomb_masked_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(o1, o2, o3, a, x, b, y, n, int64_t(6) * np * TILE, tprob,
                                                            mask);
}
template <typename R>
void launch_lincomb3(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n, cudaStream_t s) {
  lincomb_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(o1, o2, o3, a, x, b, y, n);
}

#define CMCG_DISPATCH_Q(q, KERNEL, ...)                                             \
  do {                                                                              \
    if ((q) == 1) KERNEL<1, R><<<bt.nblk, DOT_THREADS, 0, s>>>(__VA_ARGS__);        \
    else if ((q) == 2) KERNEL<2, R><<<bt.nblk, DOT_THREADS, 0, s>>>(__VA_ARGS__);   \
    else KERNEL<3, R><<<bt.nblk, DOT_THREADS, 0, s>>>(__VA_ARGS__);                 \
  } while (0)

template <typename R>
void launch_cg_after_adjoint(int q, const R* Uw, const R* WT, R* A, const R* D, const double* wdot, double* partials,
                             const BlockTable& bt, const int32_t* pactive, cudaStream_t s) {
  CMCG_DISPATCH_Q(q, cg_after_adjoint_kernel, Uw, WT, A, D, wdot, partials, bt, pactive);
}
template <typename R>
void launch_cg_update(int q, R* U0, R* Rv, const R* D, const R* A, const double* wdot, const Scalars* sc,
                      double* partials, const BlockTable& bt, const int32_t* pactive, cudaStream_t s) {
  CMCG_DISPATCH_Q(q, cg_update_kernel, U0, Rv, D, A, wdot, sc, partials, bt, pactive);
}
template <typename R>
void launch_dot(int q, const R* X, const R* Y, const double* wdot, double* partials, const BlockTable& bt,
                cudaStream_t s) {
  CMCG_DISPATCH_Q(q, dot_kernel, X, Y, wdot, partials, bt);
}
template <typename R>
void launch_scatter_rows(R* dst_re, R* dst_im, const double* src_re, const double* src_im, const int64_t* tet,
                         int64_t count, int np, cudaStream_t s) {
  if (count <= 0) return;
  scatter_rows_kernel<R><<<grid_for(count * 6 * np, 256), 256, 0, s>>>(dst_re, dst_im, src_re, src_im, tet, count,
                                                                         6 * np);
}
template <typename R>
void launch_halo(R* v, const int64_t* dst, const int64_t* src, int64_t n, int np, cudaStream_t s) {
  if (n <= 0) return;
  halo_kernel<R><<<grid_for(n * 6 * np, 256), 256, 0, s>>>(v, dst, src, n, 6 * np);
}
void launch_zero_wdot(double* wdot, const int64_t* tets, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  zero_wdot_kernel<<<grid_for(n, 256), 256, 0, s>>>(wdot, tets, n);
}
template <typename R>
void launch_set_gvol_item(R* gvol, int item, const double* val, const double* scale, const int32_t* e_of_i,
                          int64_t nti, cudaStream_t s) {
  if (nti <= 0) return;
  set_gvol_item_kernel<R><<<grid_for(nti, 256), 256, 0, s>>>(gvol, item, val, scale, e_of_i, nti);
}
template <typename R>
void launch_cg_direction(R* D, R* Uw, const R* Rv, const Scalars* sc, const int32_t* tprob, const int32_t* pactive,
                         int64_t n, int np, cudaStream_t s) {
  cg_direction_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(D, Uw, Rv, sc, tprob, pactive, n, int64_t(6) * np * TILE);
}
void launch_finalize(const double* partials, const BlockTable& bt, Scalars* sc, int32_t* pactive, const int32_t* used,
                     int which, double tol, cudaStream_t s) {
  finalize_kernel<<<bt.nprob, 256, 0, s>>>(partials, bt, sc, pactive, used, which, tol);
}

#define CMCG_INST(R)                                                                                                  \
  template void launch_to_internal<R>(const double*, int, int, R*, int, int, int, const int32_t*, int64_t, int,        \
                                      double, const double*, cudaStream_t);                                           \
  template void launch_to_external<R>(const R*, int, int, double*, int, int, int, const int32_t*, int64_t, int,       \
                                      cudaStream_t);                                                                  \
  template void launch_lincomb3<R>(R*, R*, R*, double, const R*, double, const R*, int64_t, cudaStream_t);             \
  template void launch_lincomb3_masked<R>(R*, R*, R*, double, const R*, double, const R*, int64_t, int,                 \
                                          const int32_t*, const int32_t*, cudaStream_t);                                \
  template void launch_cg_after_adjoint<R>(int, const R*, const R*, R*, const R*, const double*, double*,              \
                                           const BlockTable&, const int32_t*, cudaStream_t);                          \
  template void launch_cg_update<R>(int, R*, R*, const R*, const R*, const double*, const Scalars*, double*,          \
                                    const BlockTable&, const int32_t*, cudaStream_t);                                 \
  template void launch_dot<R>(int, const R*, const R*, const double*, double*, const BlockTable&, cudaStream_t);      \
  template void launch_scatter_rows<R>(R*, R*, const double*, const double*, const int64_t*, int64_t, int,        \
                                       cudaStream_t);                                                              \
  template void launch_set_gvol_item<R>(R*, int, const double*, const double*, const int32_t*, int64_t,             \
                                        cudaStream_t);                                                             \
  template void launch_halo<R>(R*, const int64_t*, const int64_t*, int64_t, int, cudaStream_t);                        \
  template void launch_cg_direction<R>(R*, R*, const R*, const Scalars*, const int32_t*, const int32_t*, int64_t,     \
                                       int, cudaStream_t);
CMCG_INST(float)
CMCG_INST(double)

}  // namespace cmcg
