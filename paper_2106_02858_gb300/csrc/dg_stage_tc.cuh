// The RK stage of dg_stage.cuh with the two dense contractions of the DG operator
// (Section 5.2.2, Eq. DG_semidiscrete / Eq. ode_system) on the 5th-generation
// tensor cores: the reference derivatives D_b F (b = r, s, t) of the own field
// and the lift LIFT . f of the face fluxes.  FP32 sweeps only; included by
// dg_stage.cuh inside its anonymous namespace, once per order.
//
// Mapping.  A CTA of 128 threads covers 64 tetrahedra (two 32-tetrahedron
// tiles); thread t is row t of every MMA and lane t of tensor memory (TMEM), and,
// as in dg_stage_kernel, threads 2k and 2k + 1 hold the electric and the magnetic
// field of one tetrahedron (each computes the other field's Phi).  Per row:
//
//   volume:  d_{c'}[(b, i)] = sum_j F_{c'}[j] D_b[i][j]      (3 MMAs chains, K = Np, N = 3 Np)
//   lift:    L_c[i]        = sum_k f_c[k] LIFT[i][k]        (3 chains, K = 4 Nfp, N = Np)
//
// with F the own field and f the face fluxes of the output field (computed on the
// CUDA cores as in dg_stage_kernel).  The A operands (per-row data) are written to
// TMEM with tcgen05.st; the B operands (reference matrices, shared by all rows)
// are staged in shared memory once per CTA by a bulk copy, in the K-major
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix, LBO = 128
// bytes between core matrices along K, SBO between groups of 8 rows).  The chain
// rule with the tetrahedron's affine factors and the curl are applied to the
// derivatives read back from TMEM, on the CUDA cores.
//
// Precision (3xTF32).  Every FP32 value x is split x = hi + lo with hi = x
// rounded to TF32 (10 explicit mantissa bits) and lo = x - hi, of which the tensor
// core reads the leading TF32 bits; a product is hi_a hi_b + lo_a hi_b + hi_a lo_b
// (the lo_a lo_b term, ~2^-22 relative, is dropped), accumulated in FP32 in TMEM.
// The reference matrices are split on the host from double (both parts rounded).
//
// Synchronisation.  One thread issues every MMA of the CTA; the six contractions
// (volume of own components 0, 1, 2, then lift of output components 0, 1, 2) use
// two TMEM buffers in turn, each with its own mbarrier, so that at most 256 TMEM
// columns are held and two CTAs can share an SM.  All waits on mbarriers are bounded (about one second of
// %globaltimer), after which the CTA records CMCG_ERR_DEVICE_TIMEOUT in a.err,
// skips the dependent work, frees its TMEM and returns.  TMEM is allocated after
// the grid-dependency wait, so a CTA that starts early under programmatic
// dependent launch never holds TMEM while the previous stage still runs; the
// bulk copy of the reference matrices is issued before that wait.

constexpr int TC_THREADS = 128;
constexpr int TC_TETS = 64;
constexpr int TC_KV = (NPQ + 7) / 8 * 8;              // volume K (nodes), padded to the MMA K of 8
constexpr int TC_KL = (4 * NFPQ + 7) / 8 * 8;         // lift K (face nodes f Nfp + jf)
// Accumulator columns.  The output nodes are split in two halves of NH, each half's columns
// one aligned block (a layout that lets a thread group own one node half):
//   volume: column of (b, i) = h VBLK + b NH + (i - h NH), h = i / NH;   N = 2 VBLK
//   lift:   column of i      = h LBLK + (i - h NH);                       N = 2 LBLK
constexpr int TC_NH = NPQ / 2;
constexpr int tc_pow2_at_least(int x) { return x <= 8 ? 8 : x <= 16 ? 16 : x <= 32 ? 32 : 64; }
constexpr int TC_VBLK = tc_pow2_at_least(3 * TC_NH);
constexpr int TC_LBLK = tc_pow2_at_least(TC_NH);
constexpr int TC_NV = 2 * TC_VBLK;                    // volume N
constexpr int TC_NL = 2 * TC_LBLK;                    // lift N
static_assert(NPQ % 2 == 0 && TC_NV % 16 == 0 && TC_NL % 16 == 0, "accumulator blocks");
__host__ __device__ constexpr int tc_vcol(int b, int i) {
  return (i / TC_NH) * TC_VBLK + b * TC_NH + (i % TC_NH);
}
__host__ __device__ constexpr int tc_lcol(int i) { return (i / TC_NH) * TC_LBLK + (i % TC_NH); }
// TMEM columns: two buffers of TC_BUF columns.  A buffer holds one component's
// contraction: its accumulator [0, N) and its A operand, hi [N, N + K) and lo
// [N + K, N + 2K) -- volume (N = NV, K = KV) or lift (N = NL, K = KL).  The six
// contractions (3 volume, then 3 lift) alternate between the buffers, so one
// component's MMAs run while the previous component's result is read.
constexpr int TC_NEED = (TC_NV + 2 * TC_KV) > (TC_NL + 2 * TC_KL) ? (TC_NV + 2 * TC_KV) : (TC_NL + 2 * TC_KL);
constexpr int TC_BUF = TC_NEED <= 32 ? 32 : TC_NEED <= 64 ? 64 : TC_NEED <= 128 ? 128 : 256;
constexpr int TC_COLS = 2 * TC_BUF;
static_assert(TC_COLS <= 256, "two CTAs per SM need at most 256 TMEM columns each");

// Reference matrices for the MMAs (B operands), split hi / lo, in the core-matrix
// layout: [BV hi | BV lo | BL hi | BL lo], BV = NV x KV, BL = NL x KL (row-major
// in (n, k) through tc_cm_offset).  Written by upload_constants.
constexpr int TC_BV_BYTES = TC_NV * TC_KV * 4;
constexpr int TC_BL_BYTES = TC_NL * TC_KL * 4;
constexpr int TC_B_BYTES = 2 * TC_BV_BYTES + 2 * TC_BL_BYTES;
__device__ __align__(128) uint32_t gTcB[TC_B_BYTES / 4];

// Byte offset of element (row n, column k) of an (rows x K) K-major operand.
__host__ __device__ constexpr int tc_cm_offset(int n, int k, int K) {
  return ((n >> 3) * (K >> 2) + (k >> 2)) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, LBO, SBO (bytes), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((addr >> 4) & 0x3FFF) | (uint64_t((lbo >> 4) & 0x3FFF) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFF) << 32) | (uint64_t(1) << 46);
}

// Instruction descriptor of kind::tf32: D f32, A and B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// Round an FP32 bit pattern to TF32 (nearest, ties away from zero).
__device__ __forceinline__ uint32_t tf32_rn(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }
// x = hi + lo with hi = x rounded to TF32 and lo = x - hi exactly (|lo| <= 2^-11 |x|); the
// tensor core reads lo's leading TF32 bits (it truncates), which keeps hi + lo within 2^-21 |x|.
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rn(__float_as_uint(x));
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void tmem_st8(uint32_t addr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(addr), "r"(v[0]),
               "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float (&f)[16]) {
  uint32_t v[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(addr)
      : "memory");
#pragma unroll
  for (int k = 0; k < 16; ++k) f[k] = __uint_as_float(v[k]);
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// One MMA D[tmem d] (+)= A[tmem a] B[smem desc b]^T, M = 128.
__device__ __forceinline__ void tc_mma(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Waits until the mbarrier completes phase `parity`; false after about one second.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t done = 0;
  const uint64_t t0 = globaltimer();
  for (;;) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (globaltimer() - t0 > 1000000000ull) return false;
  }
}

template <int MINB>
__global__ void __launch_bounds__(TC_THREADS, MINB) dg_stage_tc(const StageArgs<float> a) {
  using R = float;
  constexpr int NP = NPQ, NFP = NFPQ;
  constexpr int VS = 6 * NP * TILE;
  constexpr FaceTab FM = make_fmask(CMCG_Q);
  constexpr uint32_t IDV = tc_idesc(128, TC_NV), IDL = tc_idesc(128, TC_NL);
  grid_dep_launch();
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t gthr = (int64_t)blockIdx.x * TC_THREADS + tid;
  const int64_t gt = gthr >> 1;
  const int half = int(gthr & 1);  // 0: owns E, computes Phi_H;  1: owns H, computes Phi_E
  const int64_t tile = gt >> 5;
  const int lane = int(gt & 31);
  const bool in_range = gt < a.nti;  // warp-uniform (nti is a multiple of 32)

  __shared__ __align__(8) uint64_t bars[3];  // [0]: reference matrices loaded, [1 + b]: MMAs of buffer b
  __shared__ uint32_t tmem_base;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* sB = smem_raw;                                            // TC_B_BYTES
  R* tr = reinterpret_cast<R*>(smem_raw + TC_B_BYTES) + tid;               // trace / flux slots
  R* bs = tr + TRACE_SLOTS * TC_THREADS;                                   // base rows
  R* js = bs + 3 * NP * TC_THREADS;  // source rows (single-frequency source stages): J_re (half 1), J_im (half 0)
  const bool jpre = a.jre && a.nharm <= 0;

  int prob = 0;
  StageCoef<R> cf;
  cf.active = 0;
  if (in_range) {
    prob = a.tprob ? a.tprob[tile] : 0;
    cf = a.coef[prob];
  }
  bool live = in_range && cf.active;
  if (!__syncthreads_or(live)) return;  // CTA-uniform
  const int cOwn = half ? 3 : 0, cOut = half ? 0 : 3;
  const R sH = a.sH;
  const R sIn = half ? sH : R(1);
  const R sOut = half ? R(1) : sH;
  const R pec = half ? R(0) : R(-2);
  R G[9], sv = 0;
  int32_t code[4] = {NBR_PEC, NBR_PEC, NBR_PEC, NBR_PEC};
  R fn[4][3], fk1[4], fk2[4];
#pragma unroll
  for (int m = 0; m < 9; ++m) G[m] = 0;
#pragma unroll
  for (int f = 0; f < 4; ++f) fn[f][0] = fn[f][1] = fn[f][2] = fk1[f] = fk2[f] = 0;
  if (live) {
    const R* gv = a.gvol + tile * GV * TILE + lane;
#pragma unroll
    for (int m = 0; m < 9; ++m) G[m] = gv[m * TILE];
    sv = half ? -gv[9 * TILE] : gv[10 * TILE] * sOut;
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      code[f] = a.nbr[(tile * 4 + f) * TILE + lane];
      const R* gf = a.gface + (tile * 4 + f) * GF * TILE + lane;
      fn[f][0] = gf[0];
      fn[f][1] = gf[TILE];
      fn[f][2] = gf[2 * TILE];
      fk1[f] = gf[(3 + 2 * half) * TILE] * sOut;
      fk2[f] = gf[(4 + 2 * half) * TILE] * sOut;
    }
  }
  // The reference matrices (written only at handle creation) are copied before the grid
  // dependency: one bulk copy, completion counted in bytes on barB.
  const uint32_t barB = smem_addr(&bars[0]);
  const uint32_t barM[2] = {smem_addr(&bars[1]), smem_addr(&bars[2])};
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barB));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barM[0]));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barM[1]));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(barB), "r"(TC_B_BYTES) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(sB)),
        "l"(gTcB), "r"(TC_B_BYTES), "r"(barB)
        : "memory");
  }
  grid_dep_wait();
  if (live && a.pactive && !a.pactive[prob]) live = false;  // CG converged (written by the CG kernels)
  if (!__syncthreads_or(live)) {
    if (tid == 0) mbar_wait(barB, 0);  // the copy lands before the CTA's shared memory is released
    return;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_base)),
                 "r"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }

  // Own field, neighbour traces, base rows and (single-frequency source stages) source rows.
  R v[3][NP];
  const int64_t off = tile * VS + cOut * NP * TILE + lane;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int n = 0; n < NP; ++n) v[c][n] = R(0);
  if (live) {
    const R* vin = a.vin + tile * VS + cOwn * NP * TILE + lane;
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int n = 0; n < NP; ++n) v[c][n] = sIn * vin[(c * NP + n) * TILE];
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
          for (int c = 0; c < 3; ++c)
            cp_async_4(tr + ((f * NFP + jf) * 3 + c) * TC_THREADS, nb + (c * NP + nn) * TILE);
        }
      }
    }
    if (a.out) {
#pragma unroll
      for (int k = 0; k < 3 * NP; ++k) cp_async_4(bs + k * TC_THREADS, a.base + off + k * TILE);
    }
    if (jpre) {
      const R* src = (half ? a.jre : a.jim) + tile * (3 * NP * TILE) + lane;
#pragma unroll
      for (int k = 0; k < 3 * NP; ++k) cp_async_4(js + k * TC_THREADS, src + k * TILE);
    }
  }
  cp_async_commit();

  tc_fence_before();
  __syncthreads();  // TMEM address and mbarrier initialisation visible
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);  // this warp's TMEM lanes

  const uint32_t sb = smem_addr(sB);
  // Volume A of component c into buffer b: the own field, split hi / lo, zero-padded to KV columns.
  auto store_vol_a = [&](int b, int c) {
#pragma unroll
    for (int k0 = 0; k0 < TC_KV; k0 += 8) {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k0 + k < NP) {
          tf32_split(v[c][k0 + k], hi[k], lo[k]);
        } else {
          hi[k] = 0u;
          lo[k] = 0u;
        }
      }
      tmem_st8(trow + b * TC_BUF + TC_NV + k0, hi);
      tmem_st8(trow + b * TC_BUF + TC_NV + TC_KV + k0, lo);
    }
  };
  // Lift A of output component c into buffer b: the face fluxes (in the trace slots), split.
  auto store_lift_a = [&](int b, int c) {
#pragma unroll
    for (int k0 = 0; k0 < TC_KL; k0 += 8) {
      uint32_t hi[8], lo[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (k0 + k < 4 * NFP) {
          tf32_split(tr[((k0 + k) * 3 + c) * TC_THREADS], hi[k], lo[k]);
        } else {
          hi[k] = 0u;
          lo[k] = 0u;
        }
      }
      tmem_st8(trow + b * TC_BUF + TC_NL + k0, hi);
      tmem_st8(trow + b * TC_BUF + TC_NL + TC_KL + k0, lo);
    }
  };
  // MMAs of buffer b (thread 0): D = A_lo B_hi + A_hi B_lo + A_hi B_hi over the K steps,
  // then a commit to the buffer's mbarrier (also when skipped, so that waiters are released).
  auto issue = [&](int b, bool lift, bool go) {
    if (go) {
      const uint32_t d = tmem + b * TC_BUF;
      const uint32_t nacc = lift ? TC_NL : TC_NV;
      const int K = lift ? TC_KL : TC_KV;
      const uint32_t b0 = sb + (lift ? 2 * TC_BV_BYTES : 0);
      const uint32_t blo_off = lift ? TC_BL_BYTES : TC_BV_BYTES;
      const uint32_t sbo = uint32_t(K / 4) * 128;
      const uint32_t idesc = lift ? IDL : IDV;
#pragma unroll 1
      for (int s8 = 0; s8 < K / 8; ++s8) {
        const uint32_t ahi = d + nacc + 8 * s8, alo = ahi + K;
        const uint64_t bhi = tc_desc(b0 + 256 * s8, 128, sbo);
        const uint64_t blo = tc_desc(b0 + blo_off + 256 * s8, 128, sbo);
        tc_mma(d, alo, bhi, idesc, s8 > 0 ? 1u : 0u);
        tc_mma(d, ahi, blo, idesc, 1u);
        tc_mma(d, ahi, bhi, idesc, 1u);
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(barM[b])
                 : "memory");
  };
  // All A operands written and all accumulator reads done before thread 0 issues MMAs.
  auto handoff = [&](bool ok_in) -> bool {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    tc_fence_before();
    const bool r = __syncthreads_and(ok_in);
    tc_fence_after();
    return r;
  };
  R phi[3][NP];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int i = 0; i < NP; ++i) phi[c][i] = R(0);
  // Volume result of own component cp (buffer b): derivatives along r, s, t, chain rule, curl.
#pragma unroll
  for (int m = 0; m < 9; ++m) G[m] *= sv;  // the material factor of Phi, folded into the chain rule
  auto read_vol = [&](int b, int cp) {
    float d[TC_NV];
#pragma unroll
    for (int k0 = 0; k0 < TC_NV; k0 += 16) {
      float t16[16];
      tmem_ld16(trow + b * TC_BUF + k0, t16);
#pragma unroll
      for (int k = 0; k < 16; ++k) d[k0 + k] = t16[k];
    }
    // curl F: component 0 = d1 F2 - d2 F1, 1 = d2 F0 - d0 F2, 2 = d0 F1 - d1 F0
    const int ap = cp == 0 ? 2 : cp == 1 ? 0 : 1;   // axis whose derivative enters with +
    const int am = cp == 0 ? 1 : cp == 1 ? 2 : 0;   // axis whose derivative enters with -
    const int cpl = cp == 0 ? 1 : cp == 1 ? 2 : 0;  // output component receiving + d_ap F_cp
    const int cmi = cp == 0 ? 2 : cp == 1 ? 0 : 1;  // output component receiving - d_am F_cp
    // (G carries the material factor sv; each derivative is accumulated into Phi as an FMA chain)
#pragma unroll
    for (int i = 0; i < NP; ++i) {
      const R d0 = d[tc_vcol(0, i)], d1 = d[tc_vcol(1, i)], d2 = d[tc_vcol(2, i)];
      phi[cpl][i] = fmaf(G[2 * 3 + ap], d2, fmaf(G[1 * 3 + ap], d1, fmaf(G[0 * 3 + ap], d0, phi[cpl][i])));
      phi[cmi][i] = fmaf(-G[2 * 3 + am], d2, fmaf(-G[1 * 3 + am], d1, fmaf(-G[0 * 3 + am], d0, phi[cmi][i])));
    }
  };
  auto read_lift = [&](int b, int c) {
    float l[TC_NL];
#pragma unroll
    for (int k0 = 0; k0 < TC_NL; k0 += 16) {
      float t16[16];
      tmem_ld16(trow + b * TC_BUF + k0, t16);
#pragma unroll
      for (int k = 0; k < 16; ++k) l[k0 + k] = t16[k];
    }
#pragma unroll
    for (int i = 0; i < NP; ++i) phi[c][i] += l[tc_lcol(i)];
  };

  // Volume contractions of components 0 and 1 (buffers 0, 1).
  store_vol_a(0, 0);
  store_vol_a(1, 1);
  asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
  tc_fence_before();
  __syncthreads();
  bool okB = true;  // thread 0: the reference matrices arrived
  if (tid == 0) {
    tc_fence_after();
    okB = mbar_wait(barB, 0);
    issue(0, false, okB);
    issue(1, false, okB);
  }

  // Face fluxes (CUDA cores, overlapping the volume MMAs), stored over the trace slots.
  cp_async_wait_all();
#pragma unroll
  for (int f = 0; f < 4; ++f) {
    const R n0 = fn[f][0], n1 = fn[f][1], n2 = fn[f][2];
    const R k2 = fk2[f];
    const R m0 = fk1[f] * n0, m1 = fk1[f] * n1, m2 = fk1[f] * n2;  // k1 n, once per face
    const bool interior = code[f] >= 0;
    const R bscale = code[f] == NBR_PEC ? pec : R(-1);
#pragma unroll
    for (int jf = 0; jf < NFP; ++jf) {
      const int own = FM.v[f][jf];
      R X[3], Y[3];
      // both jumps formed and one selected: one code path per face node (the trace slots of a
      // boundary face hold stale values, which the selection discards)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const R xi = sIn * tr[((f * NFP + jf) * 3 + c) * TC_THREADS] - v[c][own];
        const R xb = bscale * v[c][own];
        X[c] = interior ? xi : xb;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Y[c] = __shfl_xor_sync(0xffffffffu, X[c], 1);
      const R nY = n0 * Y[0] + n1 * Y[1] + n2 * Y[2];
      tr[((f * NFP + jf) * 3 + 0) * TC_THREADS] = (m1 * X[2] - m2 * X[1]) + k2 * (Y[0] - n0 * nY);
      tr[((f * NFP + jf) * 3 + 1) * TC_THREADS] = (m2 * X[0] - m0 * X[2]) + k2 * (Y[1] - n1 * nY);
      tr[((f * NFP + jf) * 3 + 2) * TC_THREADS] = (m0 * X[1] - m1 * X[0]) + k2 * (Y[2] - n2 * nY);
    }
  }

  // Component 0's result, then component 2 into buffer 0; components 1 and 2's results.
  // Buffer 0 completes phases 0, 1 (volume) and 2, 3 (lift), buffer 1 phases 0 and 1.
  bool ok = mbar_wait(barM[0], 0);
  ok = __syncthreads_and(ok && okB);
  tc_fence_after();
  if (ok) read_vol(0, 0);
  store_vol_a(0, 2);
  ok = handoff(ok);
  if (tid == 0) issue(0, false, ok);
  ok = mbar_wait(barM[1], 0) && ok;
  tc_fence_after();
  if (ok) read_vol(1, 1);
  ok = mbar_wait(barM[0], 1) && ok;
  tc_fence_after();
  if (ok) {
    read_vol(0, 2);
  }

  // Lift contractions: output components 0 and 1 (buffers 0, 1), then 2 into buffer 0.
  store_lift_a(0, 0);
  store_lift_a(1, 1);
  ok = handoff(ok);
  if (tid == 0) {
    issue(0, true, ok);
    issue(1, true, ok);
  }
  ok = mbar_wait(barM[0], 0) && ok;
  tc_fence_after();
  if (ok) read_lift(0, 0);
  store_lift_a(0, 2);
  ok = handoff(ok);
  if (tid == 0) issue(0, true, ok);
  ok = mbar_wait(barM[1], 1) && ok;
  tc_fence_after();
  if (ok) read_lift(1, 1);
  ok = mbar_wait(barM[0], 1) && ok;
  tc_fence_after();
  if (ok) read_lift(0, 2);
  // Free TMEM (every thread's TMEM reads are complete).
  tc_fence_before();
  ok = __syncthreads_and(ok);
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_COLS));
  }
  if (!ok) {
    if (tid == 0 && a.err) atomicOr(a.err, 1);
    return;
  }
  if (!live) return;

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
        const int k = (c * NP + n) * TC_THREADS;
        phi[c][n] += cf.s_cos * js[k] - cf.s_sin * js[k - 1];
      }
  } else if (half && a.jre) {
    add_source<R, NP>(phi, a, cf, tile, lane, 0);
  }
  if (a.bre) {  // impedance-face data on this thread's output rows (source sweeps only)
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
        a.out[o] = bs[(c * NP + n) * TC_THREADS] + cf.c_out * phi[c][n];
      }
  }
}

// Dynamic shared memory of dg_stage_tc: reference matrices, trace slots, base rows,
// and the prefetched source rows of single-frequency source stages (src = true).
constexpr size_t tc_smem(bool src) {
  return size_t(TC_B_BYTES) + size_t(TRACE_SLOTS + (src ? 6 : 3) * NPQ) * TC_THREADS * sizeof(float);
}
// Resident CTAs per SM that the TMEM columns allow (512 per SM).
constexpr int TC_MINB = 2;

// The MMA operands of the reference matrices, split hi / lo from double, in the
// core-matrix layout of tc_cm_offset.
void tc_upload_reference(const RefMats& rm) {
  const int np = rm.np, nfp = rm.nfp;
  std::vector<uint32_t> buf(TC_B_BYTES / 4, 0u);
  auto rn = [](double x) -> uint32_t {  // round to TF32 (nearest) through FP32
    const float f = static_cast<float>(x);
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return (u + 0x1000u) & 0xFFFFE000u;
  };
  auto put = [&](int base_bytes, int n, int k, int K, double x) {
    const uint32_t hi = rn(x);
    float fh;
    std::memcpy(&fh, &hi, 4);
    const uint32_t lo = rn(x - double(fh));
    buf[(base_bytes + tc_cm_offset(n, k, K)) / 4] = hi;
    buf[(base_bytes + (base_bytes == 0 ? TC_BV_BYTES : TC_BL_BYTES) + tc_cm_offset(n, k, K)) / 4] = lo;
  };
  const std::vector<double>* D[3] = {&rm.Dr, &rm.Ds, &rm.Dt};
  for (int b = 0; b < 3; ++b)
    for (int i = 0; i < np; ++i)
      for (int j = 0; j < np; ++j) put(0, tc_vcol(b, i), j, TC_KV, (*D[b])[size_t(i) * np + j]);
  for (int i = 0; i < np; ++i)
    for (int k = 0; k < 4 * nfp; ++k) put(2 * TC_BV_BYTES, tc_lcol(i), k, TC_KL, rm.LIFT[size_t(i) * 4 * nfp + k]);
  cudaMemcpyToSymbol(gTcB, buf.data(), buf.size() * 4);
}
