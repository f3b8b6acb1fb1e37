// Host-side mesh set-up: validation, face matching, geometry, CFL step
// (Eq. cfl), and the device layout.
//
// Device layout.  Tetrahedra are renumbered internally: they are grouped by
// shape class (identical edge vectors up to 1e-9 relative, e.g. the six Kuhn
// tetrahedra of a Cartesian mesh), each group is sorted by centroid (z, then y,
// then x on a grid of a quarter of the smallest edge), and each group is padded
// to a multiple of 32.  A tile of 32 consecutive internal tetrahedra is one warp
// of the stage kernel; every per-tetrahedron quantity is stored [tile][item][lane]
// so that a warp's loads are contiguous, and within a group neighbouring
// tetrahedra across a given face sit in neighbouring lanes.  Meshes with more
// than 64 shape classes form a single group sorted by centroid.  Padding
// tetrahedra have zero geometry, PEC faces and zero weights, so their fields
// stay zero.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>
#include <unordered_map>

#include "common.h"

namespace cmcg {
namespace {

struct FaceKey {
  int32_t a, b, c;
  bool operator==(const FaceKey& o) const { return a == o.a && b == o.b && c == o.c; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = (uint64_t)(uint32_t)k.a * 0x9E3779B97F4A7C15ull;
    h ^= (uint64_t)(uint32_t)k.b + 0x7F4A7C15ull + (h << 6) + (h >> 2);
    h ^= (uint64_t)(uint32_t)k.c + 0x9E3779B9ull + (h << 6) + (h >> 2);
    return (size_t)h;
  }
};

int fail(std::string* why, const std::string& msg, int code) {
  if (why) *why = msg;
  return code;
}

}  // namespace

bool match_faces(const cmcg_mesh* mesh, std::vector<int64_t>* nb_out) {
  const int64_t nt = mesh->nt;
  const int32_t* T = mesh->tets;
  std::vector<int64_t>& nb = *nb_out;
  nb.assign(size_t(4 * nt), -1);
  std::unordered_map<FaceKey, int64_t, FaceKeyHash> map;
  map.reserve(size_t(4 * nt));
  for (int64_t k = 0; k < nt; ++k)
    for (int f = 0; f < 4; ++f) {
      int32_t g[3] = {T[4 * k + FACE_VERTS[f][0]], T[4 * k + FACE_VERTS[f][1]], T[4 * k + FACE_VERTS[f][2]]};
      std::sort(g, g + 3);
      FaceKey key{g[0], g[1], g[2]};
      auto it = map.find(key);
      if (it == map.end()) {
        map.emplace(key, 4 * k + f);
      } else {
        if (it->second < 0) return false;
        nb[4 * k + f] = it->second;
        nb[it->second] = 4 * k + f;
        it->second = -1;
      }
    }
  return true;
}

int validate_and_layout(const cmcg_mesh* mesh, const double* eps, const double* mu, double omega,
                        const cmcg_options* opt, HostLayout* out, bool build_layout, std::string* why) {
  if (!mesh || !eps || !mu || !opt) return fail(why, "null argument", CMCG_ERR_INVALID_ARG);
  if (mesh->nt <= 0 || mesh->nv < 4 || !mesh->verts || !mesh->tets || !mesh->face_tags)
    return fail(why, "empty mesh or null mesh array", CMCG_ERR_INVALID_ARG);
  if (mesh->nt > (int64_t(1) << 26) - 64 * TILE)
    return fail(why, "too many tetrahedra (limit 2^26 - 2048)", CMCG_ERR_INVALID_ARG);
  if (!(omega > 0) || !std::isfinite(omega)) return fail(why, "omega must be positive", CMCG_ERR_INVALID_ARG);
  const int q = opt->order;
  if (q < 1 || q > 3) return fail(why, "order must be 1, 2 or 3", CMCG_ERR_INVALID_ARG);
  if (opt->precision != CMCG_FP64 && opt->precision != CMCG_FP32)
    return fail(why, "bad precision", CMCG_ERR_INVALID_ARG);
  if (opt->flux != CMCG_FLUX_UPWIND && opt->flux != CMCG_FLUX_CENTRED) return fail(why, "bad flux", CMCG_ERR_INVALID_ARG);
  if (opt->steps_per_period < 0) return fail(why, "steps_per_period < 0", CMCG_ERR_INVALID_ARG);
  if (opt->stage_variant < 0) return fail(why, "stage_variant < 0", CMCG_ERR_INVALID_ARG);
  if (opt->stage_overlap < 0 || opt->stage_overlap > 2) return fail(why, "stage_overlap not in 0..2", CMCG_ERR_INVALID_ARG);
  if (opt->launch_graphs < 0 || opt->launch_graphs > 2) return fail(why, "launch_graphs not in 0..2", CMCG_ERR_INVALID_ARG);
  const int64_t nt = mesh->nt, nv = mesh->nv;
  const double* Xv = mesh->verts;
  const int32_t* T = mesh->tets;
  for (int64_t i = 0; i < 3 * nv; ++i)
    if (!std::isfinite(Xv[i])) return fail(why, "non-finite vertex coordinate", CMCG_ERR_INVALID_ARG);
  for (int64_t k = 0; k < nt; ++k) {
    if (!(eps[k] > 0) || !(mu[k] > 0) || !std::isfinite(eps[k]) || !std::isfinite(mu[k]))
      return fail(why, "eps and mu must be positive and finite", CMCG_ERR_INVALID_ARG);
    for (int v = 0; v < 4; ++v) {
      if (T[4 * k + v] < 0 || T[4 * k + v] >= nv) return fail(why, "vertex index out of range", CMCG_ERR_INVALID_ARG);
      for (int w = 0; w < v; ++w)
        if (T[4 * k + v] == T[4 * k + w]) return fail(why, "repeated vertex in a tetrahedron", CMCG_ERR_INVALID_ARG);
    }
    for (int f = 0; f < 4; ++f) {
      uint8_t t = mesh->face_tags[4 * k + f];
      if (t > 2) return fail(why, "face tag must be 0, 1 or 2", CMCG_ERR_INVALID_ARG);
    }
  }

  // --- geometry (double) ------------------------------------------------------------------
  const RefMats& rm = ref_mats(q);
  std::vector<double> G(9 * nt), absdet(nt), nrm(12 * nt), area(4 * nt), cen(3 * nt);
  double rho_min = 1e300, hmin = 1e300;
  for (int64_t k = 0; k < nt; ++k) {
    const double* v0 = Xv + 3 * (int64_t)T[4 * k + 0];
    double A[3][3];  // A[d][b] = (v_{b+1} - v0)_d
    for (int b = 0; b < 3; ++b) {
      const double* vb = Xv + 3 * (int64_t)T[4 * k + b + 1];
      for (int d = 0; d < 3; ++d) A[d][b] = vb[d] - v0[d];
    }
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                 A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double scale = 0;
    for (int d = 0; d < 3; ++d)
      for (int b = 0; b < 3; ++b) scale = std::max(scale, std::fabs(A[d][b]));
    if (!(std::fabs(det) > 1e-14 * scale * scale * scale)) return fail(why, "degenerate tetrahedron", CMCG_ERR_INVALID_ARG);
    // inverse: Ginv[b][a] = d r_b / d x_a
    double inv[3][3];
    inv[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
    inv[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    inv[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    inv[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
    inv[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    inv[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    inv[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
    inv[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    inv[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) G[9 * k + 3 * b + a] = inv[b][a];
    absdet[k] = std::fabs(det);
    // grad lambda_f: f = 1..3 rows of inv, f = 0 minus their sum; outward normal = -grad / |grad|
    double gl[4][3];
    for (int a = 0; a < 3; ++a) {
      gl[1][a] = inv[0][a];
      gl[2][a] = inv[1][a];
      gl[3][a] = inv[2][a];
      gl[0][a] = -(inv[0][a] + inv[1][a] + inv[2][a]);
    }
    double atot = 0;
    for (int f = 0; f < 4; ++f) {
      double len = std::sqrt(gl[f][0] * gl[f][0] + gl[f][1] * gl[f][1] + gl[f][2] * gl[f][2]);
      for (int a = 0; a < 3; ++a) nrm[12 * k + 3 * f + a] = -gl[f][a] / len;
      area[4 * k + f] = 0.5 * absdet[k] * len;  // 3 |K| |grad lambda_f|, |K| = |det| / 6
      atot += area[4 * k + f];
    }
    double rho = absdet[k] / atot;  // 6 |K| / |dK|
    rho_min = std::min(rho_min, std::sqrt(mu[k] * eps[k]) * rho);
    for (int d = 0; d < 3; ++d) {
      double c = 0.25 * (v0[d] + Xv[3 * (int64_t)T[4 * k + 1] + d] + Xv[3 * (int64_t)T[4 * k + 2] + d] +
                         Xv[3 * (int64_t)T[4 * k + 3] + d]);
      cen[3 * k + d] = c;
    }
    hmin = std::min(hmin, std::cbrt(absdet[k]));
  }

  // --- face matching -------------------------------------------------------------------------
  std::vector<int64_t> nb;  // neighbour (tet*4 + face)
  if (!match_faces(mesh, &nb)) return fail(why, "a face is shared by more than two tetrahedra", CMCG_ERR_NONCONFORMING_MESH);
  for (int64_t kf = 0; kf < 4 * nt; ++kf) {
    uint8_t t = mesh->face_tags[kf];
    if (nb[kf] >= 0 && t != CMCG_TAG_INTERIOR)
      return fail(why, "boundary tag on a face shared by two tetrahedra", CMCG_ERR_NONCONFORMING_MESH);
    if (nb[kf] < 0 && t == CMCG_TAG_INTERIOR)
      return fail(why, "unshared face without a PEC or impedance tag", CMCG_ERR_NONCONFORMING_MESH);
  }

  // --- steps per period (Eq. cfl) ---------------------------------------------------------------
  // Section 5.3 prints c_1 = 0.24 (RK2) and c_3 = 0.12 (RK4) from 2D experiments.  In 3D the
  // printed c_1 is not stable (on Kuhn meshes of 8^3 cubes and more with permittivity jumps one
  // RK2 period multiplies a mode by 10 and more), so P1 uses half of it; P2 / P3 use 0.12.
  const double c_q = opt->c_q > 0 ? opt->c_q : 0.12;
  const double Tper = 2.0 * M_PI / omega;
  int steps = opt->steps_per_period;
  if (steps <= 0) {
    double s = std::ceil(Tper / (c_q * rho_min));
    if (!(s < 2e9)) return fail(why, "time step too small", CMCG_ERR_INVALID_ARG);
    steps = std::max(1, int(s));
  }
  if (out) {
    out->steps = steps;
    out->T = Tper;
    out->dt = Tper / steps;
    out->rho_min = rho_min;
    out->q = q;
    out->np = rm.np;
    out->nt = nt;
  }
  if (!build_layout) return CMCG_OK;

  // --- shape classes and internal order -----------------------------------------------------------
  std::vector<int> cls(nt, 0);
  int ngroups = 1;
  {
    std::map<std::array<int64_t, 9>, int> classes;
    bool too_many = false;
    for (int64_t k = 0; k < nt && !too_many; ++k) {
      const double* v0 = Xv + 3 * (int64_t)T[4 * k];
      std::array<int64_t, 9> key;
      for (int b = 0; b < 3; ++b)
        for (int d = 0; d < 3; ++d)
          key[3 * b + d] = (int64_t)std::llround((Xv[3 * (int64_t)T[4 * k + b + 1] + d] - v0[d]) / (1e-9 * hmin));
      auto it = classes.find(key);
      if (it == classes.end()) {
        if ((int)classes.size() >= 64) {
          too_many = true;
          break;
        }
        it = classes.emplace(key, (int)classes.size()).first;
      }
      cls[k] = it->second;
    }
    if (too_many) std::fill(cls.begin(), cls.end(), 0);
    else ngroups = (int)classes.size();
  }
  std::vector<int64_t> order(nt);
  for (int64_t k = 0; k < nt; ++k) order[k] = k;
  const double gq = 0.25 * hmin;
  auto qc = [&](int64_t k, int d) { return (int64_t)std::floor(cen[3 * k + d] / gq); };
  std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (cls[a] != cls[b]) return cls[a] < cls[b];
    int64_t za = qc(a, 2), zb = qc(b, 2);
    if (za != zb) return za < zb;
    int64_t ya = qc(a, 1), yb = qc(b, 1);
    if (ya != yb) return ya < yb;
    int64_t xa = qc(a, 0), xb = qc(b, 0);
    if (xa != xb) return xa < xb;
    return a < b;
  });
  std::vector<int32_t> ext_of_int;
  ext_of_int.reserve(nt + 32 * ngroups);
  for (int64_t i = 0; i < nt; ++i) {
    ext_of_int.push_back((int32_t)order[i]);
    bool end_group = (i + 1 == nt) || cls[order[i + 1]] != cls[order[i]];
    if (end_group)
      while (ext_of_int.size() % TILE) ext_of_int.push_back(-1);
  }
  const int64_t nti = (int64_t)ext_of_int.size();
  const int64_t ntiles = nti / TILE;
  std::vector<int32_t> int_of_ext(nt);
  for (int64_t i = 0; i < nti; ++i)
    if (ext_of_int[i] >= 0) int_of_ext[ext_of_int[i]] = (int32_t)i;

  // --- device-layout arrays --------------------------------------------------------------------
  out->ngroups = ngroups;
  out->nti = nti;
  out->ntiles = ntiles;
  out->gvol.assign(ntiles * GV * TILE, 0.0);
  out->gface.assign(ntiles * 4 * GF * TILE, 0.0);
  out->nbr.assign(ntiles * 4 * TILE, NBR_PEC);
  out->wdot.assign(ntiles * 2 * TILE, 0.0);
  const bool centred = opt->flux == CMCG_FLUX_CENTRED;
  for (int64_t i = 0; i < nti; ++i) {
    const int64_t e = ext_of_int[i];
    if (e < 0) continue;
    const int64_t tile = i / TILE, lane = i % TILE;
    auto gv = [&](int item) -> double& { return out->gvol[(tile * GV + item) * TILE + lane]; };
    for (int m = 0; m < 9; ++m) gv(m) = G[9 * e + m];
    gv(9) = 1.0 / eps[e];
    gv(10) = 1.0 / mu[e];
    out->wdot[(tile * 2 + 0) * TILE + lane] = absdet[e] * eps[e];
    out->wdot[(tile * 2 + 1) * TILE + lane] = absdet[e] * mu[e];
    const double Zm = std::sqrt(mu[e] / eps[e]), Ym = 1.0 / Zm;
    for (int f = 0; f < 4; ++f) {
      auto gf = [&](int item) -> double& { return out->gface[((tile * 4 + f) * GF + item) * TILE + lane]; };
      for (int a = 0; a < 3; ++a) gf(a) = nrm[12 * e + 3 * f + a];
      const double fscale = area[4 * e + f] / rm.face_ref_area[f] / absdet[e];
      double Zp = Zm, Yp = Ym;
      int32_t code;
      const int64_t nkf = nb[4 * e + f];
      if (nkf >= 0) {
        const int64_t en = nkf / 4;
        const int fn = int(nkf % 4);
        Zp = std::sqrt(mu[en] / eps[en]);
        Yp = 1.0 / Zp;
        // perm: own face-local vertex s is neighbour face-local vertex sigma[s]
        int sigma[3];
        for (int s = 0; s < 3; ++s) {
          int32_t gs = T[4 * e + FACE_VERTS[f][s]];
          sigma[s] = -1;
          for (int s2 = 0; s2 < 3; ++s2)
            if (T[4 * en + FACE_VERTS[fn][s2]] == gs) sigma[s] = s2;
        }
        int p = -1;
        for (int pp = 0; pp < 6; ++pp)
          if (PERMS[pp][0] == sigma[0] && PERMS[pp][1] == sigma[1] && PERMS[pp][2] == sigma[2]) p = pp;
        if (p < 0) return fail(why, "face vertices do not match", CMCG_ERR_NONCONFORMING_MESH);
        code = (int32_t(int_of_ext[en]) << 5) | (fn << 3) | p;
      } else {
        code = mesh->face_tags[4 * e + f] == CMCG_TAG_PEC ? NBR_PEC : NBR_IMP;
      }
      out->nbr[(tile * 4 + f) * TILE + lane] = code;
      // E-rows flux  fE = aE (dE - n (n.dE)) - bE n x dH,  H-rows flux  fH = bH n x dE + aH (dH - n (n.dH))
      // with aE = fscale / (eps (Z- + Z+)), bE = Z+ aE, aH = fscale / (mu (Y- + Y+)), bH = Y+ aH.
      // Stored per half of the thread pair: (k1, k2) = (bH, aH) for the thread that owns E and
      // computes Phi_H, (-bE, aE) for the thread that owns H and computes Phi_E.
      const double aE = fscale / eps[e] / (Zm + Zp), aH = fscale / mu[e] / (Ym + Yp);
      gf(3) = Yp * aH;
      gf(4) = centred ? 0.0 : aH;
      gf(5) = -Zp * aE;
      gf(6) = centred ? 0.0 : aE;
    }
  }
  out->ext_of_int = std::move(ext_of_int);
  out->int_of_ext = std::move(int_of_ext);
  return CMCG_OK;
}

}  // namespace cmcg
