// Element partition of a mesh for sharded sweeps (host only).
//
// The DG operator (Section 5.2.2, Eq. DG_semidiscrete) is element-local except for the face
// fluxes, which read the neighbour's trace.  A part of an element partition therefore needs,
// per RK stage, only the stage values of the tetrahedra across its cut faces (its ghosts), and
// CMCG (Section 2.2, Algorithm cmcg) needs, per CG iteration, the sums of its FP64 inner
// products over all parts.  This file builds the partition (slabs along an axis) and, per
// part, the local mesh (owned tetrahedra, then ghosts) with the owner of every ghost; the
// library's sharded handles (cmcg_create_sharded) and any multi-process driver use the same
// plan.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "common.h"

namespace cmcg {

int shard_plan(const cmcg_mesh* mesh, const std::vector<int64_t>& nb, const int32_t* part, int nparts, int p,
               ShardPlan* out) {
  const int64_t nt = mesh->nt;
  ShardPlan& S = *out;
  S = ShardPlan();
  // index of each tetrahedron within its part's owned list (owned lists are in global order)
  std::vector<int64_t> count(static_cast<size_t>(nparts), 0);
  std::vector<int32_t> local_in_owner(static_cast<size_t>(nt));
  for (int64_t k = 0; k < nt; ++k) local_in_owner[size_t(k)] = int32_t(count[size_t(part[k])]++);
  std::vector<int32_t> local_of(static_cast<size_t>(nt), -1);
  for (int64_t k = 0; k < nt; ++k)
    if (part[k] == p) {
      local_of[size_t(k)] = int32_t(S.global_of_local.size());
      S.global_of_local.push_back(int32_t(k));
    }
  S.n_owned = int64_t(S.global_of_local.size());
  std::vector<int32_t> ghosts;
  for (int64_t i = 0; i < S.n_owned; ++i) {
    const int64_t k = S.global_of_local[size_t(i)];
    for (int f = 0; f < 4; ++f) {
      const int64_t n = nb[size_t(4 * k + f)];
      if (n >= 0 && part[n / 4] != p) ghosts.push_back(int32_t(n / 4));
    }
  }
  std::sort(ghosts.begin(), ghosts.end());
  ghosts.erase(std::unique(ghosts.begin(), ghosts.end()), ghosts.end());
  for (int32_t k : ghosts) {
    local_of[size_t(k)] = int32_t(S.global_of_local.size());
    S.global_of_local.push_back(k);
    S.ghost_owner_part.push_back(part[k]);
    S.ghost_owner_local.push_back(local_in_owner[size_t(k)]);
  }
  const size_t nl = S.global_of_local.size();
  S.local_tags.assign(4 * nl, CMCG_TAG_INTERIOR);
  for (size_t i = 0; i < nl; ++i) {
    const int64_t k = S.global_of_local[i];
    for (int f = 0; f < 4; ++f) {
      const int64_t n = nb[size_t(4 * k + f)];
      if (n < 0) S.local_tags[4 * i + f] = mesh->face_tags[4 * k + f];
      else if (local_of[size_t(n / 4)] < 0) S.local_tags[4 * i + f] = CMCG_TAG_PEC;  // a ghost's outer face
    }
  }
  return CMCG_OK;
}

}  // namespace cmcg

using namespace cmcg;

namespace {

int check_mesh_indices(const cmcg_mesh* mesh) {
  if (!mesh || mesh->nt <= 0 || mesh->nv < 4 || !mesh->verts || !mesh->tets || !mesh->face_tags)
    return CMCG_ERR_INVALID_ARG;
  for (int64_t i = 0; i < 4 * mesh->nt; ++i)
    if (mesh->tets[i] < 0 || mesh->tets[i] >= mesh->nv) return CMCG_ERR_INVALID_ARG;
  return CMCG_OK;
}

}  // namespace

extern "C" {

int cmcg_partition_slabs(const cmcg_mesh* mesh, int nparts, int axis, int32_t* part) {
  if (check_mesh_indices(mesh) || !part || axis < 0 || axis > 2 || nparts < 1 || nparts > mesh->nt)
    return CMCG_ERR_INVALID_ARG;
  const int64_t nt = mesh->nt;
  std::vector<double> key(static_cast<size_t>(nt));
  for (int64_t k = 0; k < nt; ++k) {
    double c = 0;
    for (int v = 0; v < 4; ++v) c += mesh->verts[3 * int64_t(mesh->tets[4 * k + v]) + axis];
    if (!std::isfinite(c)) return CMCG_ERR_INVALID_ARG;
    key[size_t(k)] = c;
  }
  std::vector<int64_t> order(static_cast<size_t>(nt));
  std::iota(order.begin(), order.end(), int64_t(0));
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return key[size_t(a)] < key[size_t(b)]; });
  for (int64_t i = 0; i < nt; ++i) part[order[size_t(i)]] = int32_t(i * nparts / nt);
  return CMCG_OK;
}

int cmcg_shard_plan(const cmcg_mesh* mesh, const int32_t* part, int nparts, int p, int64_t* n_owned, int64_t* n_ghost,
                    int32_t* global_of_local, int32_t* ghost_owner_part, int32_t* ghost_owner_local,
                    uint8_t* local_tags) {
  if (check_mesh_indices(mesh) || !part || nparts < 1 || p < 0 || p >= nparts) return CMCG_ERR_INVALID_ARG;
  for (int64_t k = 0; k < mesh->nt; ++k)
    if (part[k] < 0 || part[k] >= nparts) return CMCG_ERR_INVALID_ARG;
  try {
    std::vector<int64_t> nb;
    if (!match_faces(mesh, &nb)) return CMCG_ERR_NONCONFORMING_MESH;
    ShardPlan S;
    int rc = shard_plan(mesh, nb, part, nparts, p, &S);
    if (rc) return rc;
    const int64_t ng = int64_t(S.ghost_owner_part.size());
    if (n_owned) *n_owned = S.n_owned;
    if (n_ghost) *n_ghost = ng;
    if (global_of_local) std::memcpy(global_of_local, S.global_of_local.data(), S.global_of_local.size() * 4);
    if (ghost_owner_part) std::memcpy(ghost_owner_part, S.ghost_owner_part.data(), size_t(ng) * 4);
    if (ghost_owner_local) std::memcpy(ghost_owner_local, S.ghost_owner_local.data(), size_t(ng) * 4);
    if (local_tags) std::memcpy(local_tags, S.local_tags.data(), S.local_tags.size());
  } catch (const std::bad_alloc&) {
    return CMCG_ERR_OUT_OF_MEMORY;
  }
  return CMCG_OK;
}

}  // extern "C"
