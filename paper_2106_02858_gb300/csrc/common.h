// Internal declarations of libcmcg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/cmcg.h"

namespace cmcg {

constexpr int TILE = 32;  // tetrahedra per tile = lanes of a warp

constexpr int np_of(int q) { return (q + 1) * (q + 2) * (q + 3) / 6; }
constexpr int nfp_of(int q) { return (q + 1) * (q + 2) / 2; }

// Face f is opposite vertex f; its vertices in this order (face-local vertex s = 0, 1, 2).
constexpr int FACE_VERTS[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

// The six permutations sigma of {0,1,2}: face-local vertex s of a tetrahedron is
// face-local vertex sigma[s] of its neighbour across that face.
constexpr int PERMS[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

// Index of lattice node (i, j, k) of order q in boundary order (k outermost, i fastest).
constexpr int lattice_index(int q, int i, int j, int k) {
  int idx = 0;
  for (int kk = 0; kk < k; ++kk) idx += (q - kk + 1) * (q - kk + 2) / 2;
  for (int jj = 0; jj < j; ++jj) idx += q - k - jj + 1;
  return idx + i;
}

// Volume node of face-local node jf of face f.  Face-local nodes enumerate the
// barycentric weights (w0, w1, w2) over the face's vertices with w2 outermost,
// w1 fastest, w0 = q - w1 - w2.
struct FaceTab {
  int v[4][10];
};
constexpr FaceTab make_fmask(int q) {
  FaceTab t{};
  for (int f = 0; f < 4; ++f) {
    int jf = 0;
    for (int w2 = 0; w2 <= q; ++w2)
      for (int w1 = 0; w1 <= q - w2; ++w1) {
        int b[4] = {0, 0, 0, 0};
        b[FACE_VERTS[f][0]] = q - w1 - w2;
        b[FACE_VERTS[f][1]] = w1;
        b[FACE_VERTS[f][2]] = w2;
        t.v[f][jf++] = lattice_index(q, b[1], b[2], b[3]);
      }
  }
  return t;
}

// Reference element of order q on the unit tetrahedron, built from a monomial
// basis and exact simplex integrals (host, double).
struct RefMats {
  int q = 0, np = 0, nfp = 0;
  std::vector<double> M, Minv, Dr, Ds, Dt;  // np x np, row-major
  std::vector<double> LIFT;                 // np x (4 nfp), face-local node order
  std::vector<int> fmask;                   // 4 x nfp
  std::vector<int> nbrnode;                 // 4 (neighbour face) x 6 (perm) x nfp
  double face_ref_area[4] = {0, 0, 0, 0};
};
const RefMats& ref_mats(int q);

// Per-tetrahedron geometry in the device layout, built on the host.
struct HostLayout {
  int q = 0, np = 0;
  int64_t nt = 0, nti = 0, ntiles = 0;
  std::vector<int32_t> ext_of_int;  // internal -> external tet (-1 = padding)
  std::vector<int32_t> int_of_ext;  // external -> internal
  std::vector<double> gvol;         // [tile][GV][32]
  std::vector<double> gface;        // [tile][4][GF][32]
  std::vector<int32_t> nbr;         // [tile][4][32]
  std::vector<double> wdot;         // [tile][2][32]: |det| eps, |det| mu
  int steps = 0;
  double dt = 0, T = 0, rho_min = 0;
  int ngroups = 0;
};
constexpr int GV = 12;  // G (9, d r_b / d x_a at [b*3+a]), 1/eps, 1/mu, sigma/eps (0 unless set)
constexpr int GF = 8;   // nx, ny, nz, bH, aH, -bE, aE, pad  (see setup.cpp)

int validate_and_layout(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                        const cmcg_options* opt, HostLayout* out, bool build_layout, std::string* why);
// Face neighbours by sorted vertex triples: (*nb)[4 k + f] = 4 k' + f' or -1 (vertex indices must
// be in range); false if a face is shared by more than two tetrahedra.
bool match_faces(const cmcg_mesh* mesh, std::vector<int64_t>* nb);

// Element partition of a mesh (host only).  Part p's local mesh lists its owned tetrahedra (in
// increasing global order) followed by its ghosts: the tetrahedra of other parts that share a
// face with an owned one (increasing global order).  A ghost face whose neighbour is not in the
// local mesh is tagged PEC there (ghost values are replaced after every stage, so those faces
// never reach an owned result).
struct ShardPlan {
  int64_t n_owned = 0;
  std::vector<int32_t> global_of_local;    // owned, then ghosts
  std::vector<int32_t> ghost_owner_part;   // per ghost
  std::vector<int32_t> ghost_owner_local;  // per ghost: its index in the owner's local numbering
  std::vector<uint8_t> local_tags;         // [n_local][4]
};
int shard_plan(const cmcg_mesh* mesh, const std::vector<int64_t>& nb, const int32_t* part, int nparts, int p,
               ShardPlan* out);

// Neighbour code: >= 0: (internal neighbour << 5) | (neighbour face << 3) | perm.
constexpr int32_t NBR_PEC = -1;
constexpr int32_t NBR_IMP = -2;

// Per-problem coefficients of one stage launch (a handle holds a batch of
// problems that advance in lockstep; each reads its own entry).
//   Phi   = src + B_sigma(vin),  src = s_cos * (jre + bre) - s_sin * (jim + bim)   (B_sigma = Sigma B Sigma when sH = -1;
//           B carries -(sigma/eps) E on the E rows when a.sigma is set)
//   out   = base + c_out Phi        (skipped if out == nullptr)
//   F    += fa vin + fb Phi         (complex weights; skipped if fre == nullptr)
// (s_cos, s_sin) are the cos / sin of the source phase at the stage time, or the
// weighted sums of them that the nested RK form of a source sweep adds per stage.
// A problem whose entry has active == 0 leaves everything untouched.
template <typename R>
struct StageCoef {
  R c_out, s_cos, s_sin, fa_re, fa_im, fb_re, fb_im;
  int32_t active;
};

// Arguments of one RK stage over all tetrahedra of all problems of a handle.
template <typename R>
struct StageArgs {
  const R* vin;
  const R* base;
  R* out;
  const R* jre;  // E-rows source / eps, [tile][3][Np][32] (null: no source)
  const R* jim;
  const R* bre;  // lifted impedance-face data, all 6 rows in the field layout (null: none)
  const R* bim;
  R* fre;        // filter accumulators (null: no filter)
  R* fim;
  R sH;          // +1 forward, -1 adjoint
  const StageCoef<R>* coef;  // [problem] for this launch
  const int32_t* tprob;      // problem of each tile (null: every tile is problem 0)
  const int32_t* pactive;    // per-problem CG activity (null: all active)
  const R* gvol;
  const R* gface;
  const int32_t* nbr;
  int64_t nti;
  int32_t* err;  // device status word: a stage kernel whose bounded wait ran out ORs in 1 (null: not recorded)
  int32_t sigma;  // nonzero: some tetrahedron has a conductivity (sigma/eps in gvol item 11)
  // Several harmonics in one sweep (nharm > 0): the source is sum_h hcs[2h] J_re,h - hcs[2h+1] J_im,h
  // with J_h = jre / jim + h * jstride (hcs: this launch's cos / sin of the harmonics at the stage time).
  int32_t nharm;
  int64_t jstride;
  const R* hcs;
};

// Kernel launchers, one translation unit per order.
// form: stage-kernel form.  FP32: 0, 1, 2 = two threads per tetrahedron with at
// least 1, 3, 4 resident 128-thread blocks per SM; 3, 4, 5 = four threads per
// tetrahedron with at least 4, 5, 6; 6 = tensor-core contractions (tcgen05,
// 3xTF32) with two threads per tetrahedron.  FP64: 0 = two threads per
// tetrahedron, 1, 2 = four threads per tetrahedron with at least 2, 3 blocks.
// pdl: launch with programmatic stream serialisation (the stage overlaps the
// previous stage's tail).
constexpr int STAGE_FORMS_F32 = 7;
constexpr int STAGE_FORM_TC = 6;
constexpr int STAGE_FORMS_F64 = 3;
template <int Q, typename R>
void launch_stage(const StageArgs<R>& a, cudaStream_t s, int form, bool pdl);
template <int Q>
void upload_constants(const RefMats& rm);

// Vector kernels (vec.cu).
struct Scalars {
  double rr, rr_new, dA, alpha, beta, rr0;
  int status;
  int iters;
};

// Blocks of the problem-aligned reductions: block b covers internal tets
// [tet0[b], tet0[b] + ntet[b]) of problem prob[b]; problem p owns blocks
// [pb0[p], pb0[p + 1]).
struct BlockTable {
  const int64_t* tet0;
  const int32_t* ntet;
  const int32_t* prob;
  const int32_t* pb0;
  int nblk;
  int nprob;
  int coupled;  // nonzero: the problems are the parts of one sharded problem; every problem's
                // scalars are the sums over all blocks (the all-reduce of a sharded CG)
};
constexpr int DOT_THREADS = 128;

// Layout conversion over (tet, c in [0, cnt), node):
//   internal [tile][ncomp_in][np][32] at component c_in0 + c  <->  external [tet][ncomp_ext][np] at c_ext0 + c.
// to_internal multiplies by scale (and by per_tet[e] if non-null); padding tets get 0.
template <typename R>
void launch_to_internal(const double* ext, int ncomp_ext, int c_ext0, R* in, int ncomp_in, int c_in0, int cnt,
                        const int32_t* ext_of_int, int64_t nti, int np, double scale, const double* per_tet,
                        cudaStream_t s);
template <typename R>
void launch_to_external(const R* in, int ncomp_in, int c_in0, double* ext, int ncomp_ext, int c_ext0, int cnt,
                        const int32_t* ext_of_int, int64_t nti, int np, cudaStream_t s);
// o1 = o2 = o3 = a x + b y (null outputs skipped, y may be null).
template <typename R>
void launch_lincomb3(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n, cudaStream_t s);

// The same on the tiles of the problems with mask[p] != 0 only (tprob: problem of each tile, or null).
template <typename R>
void launch_lincomb3_masked(R* o1, R* o2, R* o3, double a, const R* x, double b, const R* y, int64_t n, int np,
                            const int32_t* tprob, const int32_t* mask, cudaStream_t s);

// (eps, mu)-weighted dots and CG updates, one partial per block of the table.
template <typename R>
void launch_cg_after_adjoint(int q, const R* Uw, const R* WT, R* A, const R* D, const double* wdot, double* partials,
                             const BlockTable& bt, const int32_t* pactive, cudaStream_t s);
template <typename R>
void launch_cg_update(int q, R* U0, R* Rv, const R* D, const R* A, const double* wdot, const Scalars* sc,
                      double* partials, const BlockTable& bt, const int32_t* pactive, cudaStream_t s);
template <typename R>
void launch_dot(int q, const R* X, const R* Y, const double* wdot, double* partials, const BlockTable& bt,
                cudaStream_t s);
// Writes `count` tetrahedra's 6 Np rows (src: [count][6 Np], double) into two field vectors
// (re, im) at internal tetrahedra tet[i]; other tetrahedra are untouched.
template <typename R>
void launch_scatter_rows(R* dst_re, R* dst_im, const double* src_re, const double* src_im, const int64_t* tet,
                         int64_t count, int np, cudaStream_t s);
// Halo exchange of a sharded handle: the 6 Np values of internal tetrahedron src[i] are copied
// to internal tetrahedron dst[i] of the same field vector (a ghost receives its owner's values).
template <typename R>
void launch_halo(R* v, const int64_t* dst, const int64_t* src, int64_t n, int np, cudaStream_t s);
// wdot = 0 for the listed internal tetrahedra (ghosts do not count in the inner products).
void launch_zero_wdot(double* wdot, const int64_t* tets, int64_t n, cudaStream_t s);
// gvol item `item` of a problem's internal tetrahedra [0, nti) = val[e] * scale[e], e = e_of_i[i]
// (device arrays in the problem's external order; padding gets 0).
template <typename R>
void launch_set_gvol_item(R* gvol, int item, const double* val, const double* scale, const int32_t* e_of_i,
                          int64_t nti, cudaStream_t s);
// D = R + beta_p D and Uw = D on the tiles of active problems.
template <typename R>
void launch_cg_direction(R* D, R* Uw, const R* Rv, const Scalars* sc, const int32_t* tprob, const int32_t* pactive,
                         int64_t n, int np, cudaStream_t s);
// One block per problem sums its partials in a fixed order.
//   which 0: rr = rr0 = total, active = (used (if given) and rr0 > 0 and tol < 1)
//   which 1: dA = total, alpha = rr / dA (breakdown if dA <= 0)
//   which 2: beta = total / rr, rr = total, iters += 1, active = (sqrt(rr) > tol sqrt(rr0))
//   which 3: rr_new = total
//   which 4: as 0, for the problems with used[p] != 0 only (the others are left untouched)
// Problems with pactive[p] == 0 are left alone for which 1 and 2.
void launch_finalize(const double* partials, const BlockTable& bt, Scalars* sc, int32_t* pactive, const int32_t* used,
                     int which, double tol, cudaStream_t s);
void upload_dot_mass(int q, const double* M);

// Gauss-Legendre rule on [0, 1] (refelem.cpp).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

}  // namespace cmcg
