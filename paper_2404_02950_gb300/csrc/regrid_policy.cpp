// Regrid of a live hierarchy (Sec. 2.2-2.3) in one call: the refinement
// criteria's block masks, global (Berger-Rigoutsos style) or local
// clustering, and the rebuild of every changed level, with the paper's rule
// for falling back from local to global regrids.  The new levels' buffers
// come from the caller's allocator (the library never owns field memory).
#include <algorithm>
#include <cstring>
#include <vector>

#include "slh_internal.cuh"

namespace slh {
namespace {

long long box_cells(const slh_box& b) {
  return (long long)(b.hi[0] - b.lo[0] + 1) * (b.hi[1] - b.lo[1] + 1) * (b.hi[2] - b.lo[2] + 1);
}

long long level_cells(const slh_ctx* c, int l) {
  long long v = 0;
  for (const slh_box& b : c->lev[l].boxes) v += box_cells(b);
  return v;
}

// Give level lev the boxes (none: remove lev and every finer level), with
// buffers from the caller's allocator.
slh_status apply_level(slh_ctx* c, int lev, const std::vector<slh_box>& boxes, int itype, slh_level_alloc_fn alloc,
                       void* user) {
  if (boxes.empty()) {
    slh_status st = slh_regrid_level(c, lev, nullptr, 0, nullptr, nullptr, itype);
    if (st != SLH_OK) return st;
    if (alloc(user, lev, nullptr, 0, 0, 0, nullptr, nullptr) != 0)
      return fail(SLH_ERR_NOMEM, "regrid: the allocator refused the removal of level %d", lev);
    return SLH_OK;
  }
  int64_t total = 0, nvalid = 0;
  slh_status st = slh_level_layout(c->g, c->nslots, boxes.data(), (int32_t)boxes.size(), nullptr, nullptr, &total,
                                   &nvalid);
  if (st != SLH_OK) return st;
  void* bufs[SLH_NBUF] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  uint8_t* tags = nullptr;
  if (alloc(user, lev, boxes.data(), (int32_t)boxes.size(), total, nvalid, bufs, &tags) != 0)
    return fail(SLH_ERR_NOMEM, "regrid: the allocator failed for level %d (%lld elements)", lev, (long long)total);
  return slh_regrid_level(c, lev, boxes.data(), (int32_t)boxes.size(), bufs, tags, itype);
}

// Global regrid of the levels above `start`: the block mask of level l
// (grown tags in blocks of bf/2 cells) clustered in block units inside level
// l's boxes eroded by one block, then level l+1 rebuilt; its tags give level
// l+2.
slh_status global_regrid(slh_ctx* c, const slh_regrid_params& rp, slh_level_alloc_fn alloc, void* user) {
  const int r = c->bf / 2;
  std::vector<uint8_t> mask;
  std::vector<slh_box> parent, blocks, boxes;
  for (int l = rp.start; l < rp.max_levels - 1 && l < c->nlevels; ++l) {
    const int nb = c->lev[l].n_dom / r;
    mask.assign((size_t)nb * nb * nb, 0);
    slh_status st;
    {
      HostPhase ph(c, SLH_PROF_REGRID_TAGS);
      st = slh_tag_blocks(c, l, rp.n_error_buf, mask.data());
    }
    if (st != SLH_OK) return st;
    parent.clear();
    if (l > 0)
      for (const slh_box& b : c->lev[l].boxes) {
        slh_box p;
        for (int d = 0; d < 3; ++d) {
          p.lo[d] = b.lo[d] / r;
          p.hi[d] = (b.hi[d] + 1) / r - 1;
        }
        parent.push_back(p);
      }
    // one mask cell per block: blocking factor 2 and no further growth; the
    // boxes come back in half-blocks of level l (r cells of level l+1)
    const int dims[3] = {nb, nb, nb};
    {
      HostPhase ph(c, SLH_PROF_REGRID_CLUSTER);
      st = regrid_boxes_impl(mask.data(), dims, 2, 0, 2 * (rp.max_box / c->bf),
                             parent.empty() ? nullptr : parent.data(), (int)parent.size(), &blocks);
    }
    if (st != SLH_OK) return st;
    boxes.clear();
    for (const slh_box& b : blocks) {
      slh_box f;
      for (int d = 0; d < 3; ++d) {
        f.lo[d] = b.lo[d] * r;
        f.hi[d] = (b.hi[d] + 1) * r - 1;
      }
      boxes.push_back(f);
    }
    {
      HostPhase ph(c, SLH_PROF_REGRID_BUILD);
      st = apply_level(c, l + 1, boxes, rp.interp_type, alloc, user);
    }
    if (st != SLH_OK) return st;
    if (boxes.empty()) break;
  }
  return SLH_OK;
}

// Local regrid: every level keeps its boxes; blocks are added where the
// grown tags leave the finer level and where nesting needs them; the levels
// from the lowest changed one up are rebuilt.  added[l] receives the cells
// level l gained.
slh_status local_regrid(slh_ctx* c, const slh_regrid_params& rp, slh_level_alloc_fn alloc, void* user,
                        long long* added) {
  const int L = c->nlevels;
  for (int l = 0; l < MAX_LEVELS; ++l) added[l] = 0;
  if (L < 2) return SLH_OK;
  const int r = c->bf / 2;
  std::vector<std::vector<uint8_t>> masks(L - 1);
  std::vector<const uint8_t*> mptr(L, nullptr);
  for (int l = 0; l + 1 < L; ++l) {
    const int nb = c->lev[l].n_dom / r;
    masks[l].assign((size_t)nb * nb * nb, 0);
    HostPhase ph(c, SLH_PROF_REGRID_TAGS);
    slh_status st = slh_tag_blocks(c, l, rp.n_error_buf, masks[l].data());
    if (st != SLH_OK) return st;
    mptr[l] = masks[l].data();
  }
  std::vector<slh_box> cur;
  std::vector<int32_t> nbox(L);
  for (int l = 0; l < L; ++l) {
    cur.insert(cur.end(), c->lev[l].boxes.begin(), c->lev[l].boxes.end());
    nbox[l] = (int32_t)c->lev[l].boxes.size();
  }
  std::vector<std::vector<slh_box>> lists;
  slh_status st;
  {
    HostPhase ph(c, SLH_PROF_REGRID_CLUSTER);
    st = local_regrid_impl(L, c->n0, c->bf, mptr.data(), cur.data(), nbox.data(), &lists);
  }
  if (st != SLH_OK) return st;
  int first = -1;
  for (int l = 1; l < L; ++l) {
    long long v = 0;
    for (const slh_box& b : lists[l]) v += box_cells(b);
    added[l] = v - level_cells(c, l);
    if (added[l] > 0 && first < 0) first = l;
  }
  if (first < 0) return SLH_OK;
  for (int l = first; l < L; ++l) {
    HostPhase ph(c, SLH_PROF_REGRID_BUILD);
    if ((st = apply_level(c, l, lists[l], rp.interp_type, alloc, user)) != SLH_OK) return st;
  }
  return SLH_OK;
}

}  // namespace
}  // namespace slh

using namespace slh;

extern "C" slh_status slh_regrid(slh_ctx* c, const slh_regrid_params* rp, slh_level_alloc_fn alloc, void* user,
                                 int32_t* kind, double* frac) {
  if (!c || !rp || !alloc) return fail(SLH_ERR_INVALID_ARG, "regrid: null argument");
  if (rp->mode != SLH_REGRID_GLOBAL && rp->mode != SLH_REGRID_LOCAL && rp->mode != SLH_REGRID_AUTO)
    return fail(SLH_ERR_INVALID_ARG, "regrid: unknown mode %d", rp->mode);
  if (rp->max_levels < 1 || rp->max_levels > c->max_levels)
    return fail(SLH_ERR_INVALID_ARG, "regrid: max_levels %d outside [1,%d]", rp->max_levels, c->max_levels);
  if (rp->n_error_buf < 0) return fail(SLH_ERR_INVALID_ARG, "regrid: n_error_buf < 0");
  if (rp->max_box < c->bf || rp->max_box % c->bf)
    return fail(SLH_ERR_INVALID_ARG, "regrid: max_box must be a positive multiple of the blocking factor");
  if (rp->interp_type != 0 && rp->interp_type != 2 && rp->interp_type != 4)
    return fail(SLH_ERR_INVALID_ARG, "regrid: interp_type must be 0, 2 or 4");
  if (rp->start < 0 || (rp->start > 0 && rp->start >= c->nlevels))
    return fail(SLH_ERR_INVALID_ARG, "regrid: start level %d is not defined", rp->start);
  if (rp->mode == SLH_REGRID_AUTO && !(rp->eps_strong > 0.0 && rp->eps_weak >= 0.0 && rp->max_local >= 0))
    return fail(SLH_ERR_INVALID_ARG, "regrid: eps_strong must be > 0, eps_weak >= 0, max_local >= 0");
  if (c->nlevels < 1) return fail(SLH_ERR_STATE, "regrid: level 0 is not defined");
  // a global regrid from `start` rebuilds every level above it, so only the
  // levels up to `start` must be current; the other modes read every level
  const int need_fresh = rp->mode == SLH_REGRID_GLOBAL ? rp->start : c->nlevels - 1;
  if (c->stale_from <= need_fresh) return fail(SLH_ERR_STATE, "regrid: level %d must be regridded first", c->stale_from);
  const int L = c->nlevels;
  int k = rp->mode == SLH_REGRID_LOCAL ? SLH_REGRID_LOCAL : SLH_REGRID_GLOBAL;
  slh_regrid_params g = *rp;
  if (rp->mode == SLH_REGRID_AUTO) {
    // the volumes at the last global regrid, once per global regrid (or
    // when the number of levels changed)
    if (!c->rp_valid || c->rp_nlev != L) {
      for (int l = 0; l < MAX_LEVELS; ++l) {
        c->rp_base[l] = l < L ? (double)std::max(1LL, level_cells(c, l)) : 1.0;
        c->rp_added[l] = 0.0;
      }
      c->rp_valid = true;
      c->rp_nlev = L;
      c->rp_count = 0;
      c->rp_pending = -1;
    }
    if (c->rp_pending >= 0) {
      k = SLH_REGRID_GLOBAL;
      g.start = c->rp_pending;
    } else if (L < rp->max_levels) {
      k = SLH_REGRID_GLOBAL;
      g.start = 0;
    } else {
      k = SLH_REGRID_LOCAL;
    }
  }
  if (kind) *kind = k;
  slh_status st;
  if (k == SLH_REGRID_GLOBAL) {
    st = global_regrid(c, g, alloc, user);
    if (rp->mode == SLH_REGRID_AUTO) c->rp_valid = false;   // counters restart from the new volumes
    return st;
  }
  long long added[MAX_LEVELS];
  st = local_regrid(c, g, alloc, user, added);
  if (st != SLH_OK) return st;
  if (rp->mode == SLH_REGRID_AUTO) {
    c->rp_count += 1;
    bool strong = rp->max_local > 0 && c->rp_count >= rp->max_local;
    for (int l = 0; l < L; ++l) {
      c->rp_added[l] += (double)added[l];
      const double f = c->rp_added[l] / c->rp_base[l];
      if (frac) frac[l] = f;
      if (f >= rp->eps_strong) strong = true;
    }
    if (strong) {
      int lowest = -1;
      for (int l = 1; l < L && lowest < 0; ++l)
        if (c->rp_added[l] / c->rp_base[l] >= rp->eps_weak) lowest = l;
      c->rp_pending = lowest > 0 ? lowest - 1 : 0;
    }
  } else if (frac) {
    for (int l = 0; l < L; ++l) frac[l] = (double)added[l];
  }
  return SLH_OK;
}
