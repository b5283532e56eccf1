// Host-side regrid (Sec. 2.2-2.3): buffered tags -> blocks -> nested
// Berger-Rigoutsos style clustering -> boxes of the next finer level.
// Deterministic: every choice is made by integer comparisons with fixed tie
// breaks, so the box list depends only on the tag mask.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <thread>
#include <utility>
#include <vector>

#include "slh_internal.cuh"

namespace slh {
namespace {

struct Grid {
  int nx = 0, ny = 0, nz = 0;
  std::vector<uint8_t> v;
  Grid() = default;
  Grid(int x, int y, int z) : nx(x), ny(y), nz(z), v((size_t)x * y * z, 0) {}
  uint8_t& at(int x, int y, int z) { return v[((size_t)z * ny + y) * nx + x]; }
  uint8_t at(int x, int y, int z) const { return v[((size_t)z * ny + y) * nx + x]; }
};

// index of x + s on a periodic line of n cells (|s| <= n)
inline int wrap(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

// cube dilation with periodic wrap, one axis at a time
Grid dilate(const Grid& in, int nbuf) {
  Grid cur = in;
  for (int axis = 0; axis < 3 && nbuf > 0; ++axis) {
    Grid nxt(cur.nx, cur.ny, cur.nz);
    const int n = axis == 0 ? cur.nx : axis == 1 ? cur.ny : cur.nz;
    const int reach = std::min(nbuf, n);   // a reach of n covers the whole line
    for (int z = 0; z < cur.nz; ++z)
      for (int y = 0; y < cur.ny; ++y)
        for (int x = 0; x < cur.nx; ++x) {
          if (!cur.at(x, y, z)) continue;
          for (int s = -reach; s <= reach; ++s) {
            int p[3] = {x, y, z};
            p[axis] = wrap(p[axis] + s, n);
            nxt.at(p[0], p[1], p[2]) = 1;
          }
        }
    cur.v.swap(nxt.v);
  }
  return cur;
}

// the complement of dilate(complement of in, 1): a cell stays set when it
// and its two neighbours along each axis in turn are set (periodic wrap).
// Each pass ANDs whole rows: shifted copies of the row for x, the rows at
// y -+ 1 for y, the rows of the planes at z -+ 1 for z.
Grid erode1(Grid cur) {
  const int nx = cur.nx, ny = cur.ny, nz = cur.nz;
  Grid nxt(nx, ny, nz);
  auto row = [&](Grid& g, int y, int z) { return &g.v[((size_t)z * ny + y) * nx]; };
  for (int axis = 0; axis < 3; ++axis) {
    parallel_for(nz, (size_t)nx * ny, [&](int z) {
      for (int y = 0; y < ny; ++y) {
        const uint8_t* c = row(cur, y, z);
        uint8_t* o = row(nxt, y, z);
        if (axis == 0) {
          if (nx == 1) {
            o[0] = c[0];
            continue;
          }
          o[0] = (uint8_t)(c[0] & c[1] & c[nx - 1]);
          for (int x = 1; x < nx - 1; ++x) o[x] = (uint8_t)(c[x] & c[x - 1] & c[x + 1]);
          o[nx - 1] = (uint8_t)(c[nx - 1] & c[nx - 2] & c[0]);
        } else {
          const int n = axis == 1 ? ny : nz, pos = axis == 1 ? y : z;
          const int lo = pos == 0 ? n - 1 : pos - 1, hi = pos == n - 1 ? 0 : pos + 1;
          const uint8_t* a = axis == 1 ? row(cur, lo, z) : row(cur, y, lo);
          const uint8_t* b = axis == 1 ? row(cur, hi, z) : row(cur, y, hi);
          for (int x = 0; x < nx; ++x) o[x] = (uint8_t)(c[x] & a[x] & b[x]);
        }
      }
    });
    cur.v.swap(nxt.v);
  }
  return cur;
}

// storage of the two prefix tables, kept between calls so that a regrid does
// not page in tens of MB of fresh memory each time; 32-bit entries (a block
// grid holds fewer than 2^31 cells: checked by the caller)
thread_local std::vector<int32_t> prefix_store[2];

struct Prefix {
  int nx, ny, nz;
  std::vector<int32_t>& s;
  // one running sum per axis in turn (rows, then columns, then planes):
  // three streaming passes instead of an eight-term recurrence per cell; the
  // first two run per plane, the third per stretch of a plane, in parallel
  Prefix(const Grid& g, std::vector<int32_t>& store) : nx(g.nx), ny(g.ny), nz(g.nz), s(store) {
    const size_t plane = (size_t)(nx + 1) * (ny + 1);
    s.resize(plane * (nz + 1));
    std::fill(s.begin(), s.begin() + plane, 0);
    parallel_for(nz, plane, [&](int z) {
      int32_t* pl = &s[plane * (z + 1)];
      std::fill(pl, pl + nx + 1, 0);
      for (int y = 0; y < ny; ++y) {
        int32_t run = 0;
        const uint8_t* row = &g.v[((size_t)z * ny + y) * nx];
        int32_t* out = pl + (size_t)(y + 1) * (nx + 1);
        out[0] = 0;
        for (int x = 0; x < nx; ++x) out[x + 1] = (run += row[x]);
      }
      for (int y = 2; y <= ny; ++y) {
        int32_t* cur = pl + (size_t)y * (nx + 1) + 1;
        const int32_t* prev = cur - (nx + 1);
        for (int x = 0; x < nx; ++x) cur[x] += prev[x];
      }
    });
    const int nchunk = (int)std::min<size_t>(64, plane);
    parallel_for(nchunk, plane / nchunk * nz, [&](int c) {
      const size_t a = plane * c / nchunk, b = plane * (c + 1) / nchunk;
      for (int z = 2; z <= nz; ++z) {
        int32_t* cur = &s[plane * z];
        const int32_t* prev = cur - plane;
        for (size_t i = a; i < b; ++i) cur[i] += prev[i];
      }
    });
  }
  int64_t S(int x, int y, int z) const { return s[((size_t)z * (ny + 1) + y) * (nx + 1) + x]; }
  int64_t count(const int lo[3], const int hi[3]) const {
    const int x0 = lo[0], y0 = lo[1], z0 = lo[2], x1 = hi[0] + 1, y1 = hi[1] + 1, z1 = hi[2] + 1;
    return S(x1, y1, z1) - S(x0, y1, z1) - S(x1, y0, z1) - S(x1, y1, z0) + S(x0, y0, z1) + S(x0, y1, z0) +
           S(x1, y0, z0) - S(x0, y0, z0);
  }
};

struct BR {
  const Grid& M;
  const Prefix& PM;
  const Prefix& PA;
  int max_blocks;
  std::vector<slh_box> out;

  bool check_allowed;

  BR(const Grid& m, const Prefix& pm, const Prefix& pa, int mb, bool ca)
      : M(m), PM(pm), PA(pa), max_blocks(mb), check_allowed(ca) {}

  // tag counts of the box's planes normal to each axis, from the prefix sums
  // (O(extent) per axis instead of a pass over the box's volume)
  void signatures(const int lo[3], const int hi[3], std::vector<int64_t> sig[3]) const {
    for (int d = 0; d < 3; ++d) {
      sig[d].assign(hi[d] - lo[d] + 1, 0);
      int plo[3] = {lo[0], lo[1], lo[2]}, phi[3] = {hi[0], hi[1], hi[2]};
      for (int c = lo[d]; c <= hi[d]; ++c) {
        plo[d] = phi[d] = c;
        sig[d][c - lo[d]] = PM.count(plo, phi);
      }
    }
  }

  // shrink to the tags' bounding box; false when the box holds no tag
  bool shrink(int lo[3], int hi[3]) const {
    if (PM.count(lo, hi) == 0) return false;
    std::vector<int64_t> sig[3];
    signatures(lo, hi, sig);
    for (int d = 0; d < 3; ++d) {
      int a = 0, b = (int)sig[d].size() - 1;
      while (sig[d][a] == 0) ++a;
      while (sig[d][b] == 0) --b;
      const int base = lo[d];
      lo[d] = base + a;
      hi[d] = base + b;
    }
    return true;
  }

  void choose_cut(const int lo[3], const int hi[3], int* axis, int* cut) const {
    std::vector<int64_t> sig[3];
    signatures(lo, hi, sig);
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = hi[d] - lo[d] + 1;
    // a. zero-signature plane nearest the centre
    bool found = false;
    long bk0 = 0;
    int bd = 0, bc = 0;
    for (int d = 0; d < 3; ++d)
      for (int c = 1; c <= n[d] - 2; ++c)
        if (sig[d][c] == 0) {
          const long k0 = std::labs(2L * c - n[d]);
          if (!found || k0 < bk0 || (k0 == bk0 && (d < bd || (d == bd && c < bc)))) {
            found = true;
            bk0 = k0;
            bd = d;
            bc = c;
          }
        }
    if (found) {
      *axis = bd;
      *cut = bc;
      return;
    }
    // b. strongest sign change of the second difference
    long long bs = -1;
    for (int d = 0; d < 3; ++d) {
      if (n[d] < 4) continue;
      std::vector<long long> lap(n[d], 0);
      for (int i = 1; i <= n[d] - 2; ++i) lap[i] = sig[d][i - 1] - 2 * sig[d][i] + sig[d][i + 1];
      for (int i = 1; i <= n[d] - 3; ++i) {
        if ((lap[i] < 0 && lap[i + 1] > 0) || (lap[i] > 0 && lap[i + 1] < 0)) {
          const int c = i + 1;
          const long long st = std::llabs(lap[i + 1] - lap[i]);
          const long k0 = std::labs(2L * c - n[d]);
          bool better = false;
          if (!found || st > bs) better = true;
          else if (st == bs) {
            if (k0 < bk0) better = true;
            else if (k0 == bk0 && (d < bd || (d == bd && c < bc))) better = true;
          }
          if (better) {
            found = true;
            bs = st;
            bk0 = k0;
            bd = d;
            bc = c;
          }
        }
      }
    }
    if (found) {
      *axis = bd;
      *cut = bc;
      return;
    }
    // c. halve the longest side (lowest axis on ties)
    int d = 0;
    for (int q = 1; q < 3; ++q)
      if (n[q] > n[d]) d = q;
    *axis = d;
    *cut = n[d] / 2;
  }

  void rec(int lo_in[3], int hi_in[3]) {
    int lo[3] = {lo_in[0], lo_in[1], lo_in[2]}, hi[3] = {hi_in[0], hi_in[1], hi_in[2]};
    if (!shrink(lo, hi)) return;
    int64_t vol = 1;
    int mx = 0;
    for (int d = 0; d < 3; ++d) {
      const int n = hi[d] - lo[d] + 1;
      vol *= n;
      mx = std::max(mx, n);
    }
    const int64_t ntag = PM.count(lo, hi);
    const bool ok = 10 * ntag >= 7 * vol && mx <= max_blocks && (!check_allowed || PA.count(lo, hi) == vol);
    if (ok) {
      slh_box b;
      for (int d = 0; d < 3; ++d) {
        b.lo[d] = lo[d];
        b.hi[d] = hi[d];
      }
      out.push_back(b);
      return;
    }
    int axis = 0, cut = 0;
    choose_cut(lo, hi, &axis, &cut);
    int lhi[3] = {hi[0], hi[1], hi[2]};
    lhi[axis] = lo[axis] + cut - 1;
    int rlo[3] = {lo[0], lo[1], lo[2]};
    rlo[axis] = lo[axis] + cut;
    rec(lo, lhi);
    rec(rlo, hi);
  }
};

}  // namespace

slh_status regrid_boxes_impl(const uint8_t* tags, const int dims[3], int bf, int nbuf, int max_box,
                             const slh_box* parent, int nparent, std::vector<slh_box>* out) {
  if (!tags || !dims || !out) return fail(SLH_ERR_INVALID_ARG, "regrid: null argument");
  if (bf < 2 || (bf & (bf - 1))) return fail(SLH_ERR_INVALID_ARG, "regrid: blocking factor must be a power of two >= 2");
  if (max_box < bf || max_box % bf) return fail(SLH_ERR_INVALID_ARG, "regrid: max_box must be a positive multiple of the blocking factor");
  if (nbuf < 0) return fail(SLH_ERR_INVALID_ARG, "regrid: n_error_buf < 0");
  const int r = bf / 2;
  for (int d = 0; d < 3; ++d)
    if (dims[d] <= 0 || dims[d] % r) return fail(SLH_ERR_INVALID_ARG, "regrid: dims must be positive multiples of blocking_factor/2");
  const int bx = dims[0] / r, by = dims[1] / r, bz = dims[2] / r;
  if ((long long)(bx + 1) * (by + 1) * (bz + 1) >= (1LL << 31))
    return fail(SLH_ERR_OUT_OF_RANGE, "regrid: %d x %d x %d blocks exceed 2^31", bx, by, bz);
  const size_t cplane = (size_t)dims[0] * dims[1];
  Grid B(bx, by, bz);
  if (nbuf == 0) {
    // no growth: blocks straight from the tags
    parallel_for(bz, cplane * r, [&](int zb) {
      for (int z = zb * r; z < (zb + 1) * r; ++z)
        for (int y = 0; y < dims[1]; ++y) {
          const uint8_t* row = tags + (size_t)z * cplane + (size_t)y * dims[0];
          uint8_t* brow = &B.at(0, y / r, zb);
          for (int x = 0; x < dims[0]; ++x)
            if (row[x]) brow[x / r] = 1;
        }
    });
  } else {
    Grid T(dims[0], dims[1], dims[2]);
    for (size_t i = 0; i < T.v.size(); ++i) T.v[i] = tags[i] ? 1 : 0;
    Grid D = dilate(T, nbuf);
    for (int z = 0; z < dims[2]; ++z)
      for (int y = 0; y < dims[1]; ++y)
        for (int x = 0; x < dims[0]; ++x)
          if (D.at(x, y, z)) B.at(x / r, y / r, z / r) = 1;
  }
  Grid A(bx, by, bz);
  if (parent == nullptr || nparent == 0) {
    std::fill(A.v.begin(), A.v.end(), 1);
  } else {
    Grid P(bx, by, bz);
    for (int i = 0; i < nparent; ++i) {
      const slh_box& pb = parent[i];
      for (int d = 0; d < 3; ++d) {
        if (pb.lo[d] % r || (pb.hi[d] + 1) % r || pb.lo[d] < 0 || pb.hi[d] >= dims[d] || pb.hi[d] < pb.lo[d])
          return fail(SLH_ERR_INVALID_ARG, "regrid: parent box %d not aligned to blocking_factor/2 or outside dims", i);
      }
      const int x0 = pb.lo[0] / r, x1 = (pb.hi[0] + 1) / r, y0 = pb.lo[1] / r, y1 = (pb.hi[1] + 1) / r,
                z0 = pb.lo[2] / r, z1 = (pb.hi[2] + 1) / r;
      for (int z = z0; z < z1; ++z)
        for (int y = y0; y < y1; ++y) std::fill(&P.at(x0, y, z), &P.at(x0, y, z) + (x1 - x0), (uint8_t)1);
    }
    A = erode1(std::move(P));
  }
  Grid M(bx, by, bz);
  const size_t bplane = (size_t)bx * by;
  parallel_for(bz, bplane, [&](int z) {
    for (size_t i = z * bplane; i < (z + 1) * bplane; ++i) M.v[i] = (uint8_t)(B.v[i] & A.v[i]);
  });
  Prefix PM(M, prefix_store[0]);
  // without a parent every block is allowed: no count of allowed blocks needed
  const Prefix PA(parent == nullptr || nparent == 0 ? Grid(1, 1, 1) : A, prefix_store[1]);
  BR br(M, PM, PA, max_box / bf, parent != nullptr && nparent > 0);
  int lo[3] = {0, 0, 0}, hi[3] = {bx - 1, by - 1, bz - 1};
  br.rec(lo, hi);
  out->clear();
  for (const slh_box& b : br.out) {
    slh_box f;
    for (int d = 0; d < 3; ++d) {
      f.lo[d] = b.lo[d] * bf;
      f.hi[d] = (b.hi[d] + 1) * bf - 1;
    }
    out->push_back(f);
  }
  std::sort(out->begin(), out->end(), [](const slh_box& a, const slh_box& b) {
    if (a.lo[2] != b.lo[2]) return a.lo[2] < b.lo[2];
    if (a.lo[1] != b.lo[1]) return a.lo[1] < b.lo[1];
    return a.lo[0] < b.lo[0];
  });
  return SLH_OK;
}

}  // namespace slh

extern "C" slh_status slh_regrid_boxes(const uint8_t* tags_host, const int32_t dims[3], int32_t blocking_factor,
                                       int32_t n_error_buf, int32_t max_box, const slh_box* parent,
                                       int32_t nparent, slh_box* out, int32_t cap, int32_t* nout) {
  if (!nout) return slh::fail(SLH_ERR_INVALID_ARG, "regrid: nout is null");
  if (nparent < 0) return slh::fail(SLH_ERR_INVALID_ARG, "regrid: nparent < 0");
  int d3[3] = {dims ? dims[0] : 0, dims ? dims[1] : 0, dims ? dims[2] : 0};
  std::vector<slh_box> boxes;
  slh_status st = slh::regrid_boxes_impl(tags_host, dims ? d3 : nullptr, blocking_factor, n_error_buf, max_box,
                                         parent, nparent, &boxes);
  if (st != SLH_OK) return st;
  *nout = (int32_t)boxes.size();
  if ((int32_t)boxes.size() > cap || (!out && !boxes.empty()))
    return slh::fail(SLH_ERR_OUT_OF_RANGE, "regrid: %d boxes exceed capacity %d", (int)boxes.size(), cap);
  for (size_t i = 0; i < boxes.size(); ++i) out[i] = boxes[i];
  return SLH_OK;
}

// ---------------------------------------------------------------------------
// Local regrid (Sec. 2.3): keep every level's boxes, add blocks of the finer
// level where the grown tags are not yet covered by it, add blocks to the
// coarser levels where nesting needs them, never remove any.

namespace slh {

namespace {

struct BlockGrid {
  int n = 0;
  std::vector<uint8_t> v;
  explicit BlockGrid(int nn) : n(nn), v((size_t)nn * nn * nn, 0) {}
  uint8_t& at(int x, int y, int z) { return v[((size_t)z * n + y) * n + x]; }
  uint8_t at(int x, int y, int z) const { return v[((size_t)z * n + y) * n + x]; }
};

// blocks of `unit` cells inside the boxes (boxes given in cells of the grid's level)
slh_status cover(const slh_box* b, int nb, int unit, int shift, BlockGrid* g, const char* what) {
  for (int i = 0; i < nb; ++i) {
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = b[i].lo[d] >> shift;
      hi[d] = ((b[i].hi[d] + 1) >> shift) - 1;
      if (lo[d] % unit || (hi[d] + 1) % unit || lo[d] < 0 || hi[d] >= g->n * unit || hi[d] < lo[d])
        return fail(SLH_ERR_INVALID_ARG, "local_regrid: %s box %d not aligned or outside the domain", what, i);
    }
    for (int z = lo[2] / unit; z <= hi[2] / unit; ++z)
      for (int y = lo[1] / unit; y <= hi[1] / unit; ++y)
        for (int x = lo[0] / unit; x <= hi[0] / unit; ++x) g->at(x, y, z) = 1;
  }
  return SLH_OK;
}

}  // namespace

slh_status local_regrid_impl(int L, int n0, int bf, const uint8_t* const* masks, const slh_box* boxes,
                             const int32_t* nboxes, std::vector<std::vector<slh_box>>* out) {
  const int r = bf / 2;
  std::vector<BlockGrid> have, add;
  std::vector<int> off(L + 1, 0);
  for (int l = 0; l < L; ++l) {
    if (nboxes[l] < 0) return fail(SLH_ERR_INVALID_ARG, "local_regrid: negative box count");
    off[l + 1] = off[l] + nboxes[l];
    const int n = n0 << l;
    have.emplace_back(n / bf);
    add.emplace_back(n / bf);
    slh_status st = cover(boxes + off[l], nboxes[l], bf, 0, &have[l], "level");
    if (st != SLH_OK) return st;
  }
  // 1-3: uncovered grown tags -> new blocks of the finer level
  for (int l = 0; l + 1 < L; ++l) {
    const int nr = (n0 << l) / r;   // r-blocks of l = bf-blocks of l+1
    BlockGrid C(nr);
    slh_status st = cover(boxes + off[l + 1], nboxes[l + 1], r, 1, &C, "finer");
    if (st != SLH_OK) return st;
    if (!masks || !masks[l]) continue;
    for (size_t i = 0; i < C.v.size(); ++i)
      if (masks[l][i] && !C.v[i]) add[l + 1].v[i] = 1;
  }
  // 4: nesting closure, finest first
  for (int j = L - 1; j >= 1; --j) {
    const int nr = have[j].n;       // bf-blocks of j = r-blocks of j-1
    for (int z = 0; z < nr; ++z)
      for (int y = 0; y < nr; ++y)
        for (int x = 0; x < nr; ++x) {
          if (!have[j].at(x, y, z) && !add[j].at(x, y, z)) continue;
          for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
              for (int dx = -1; dx <= 1; ++dx) {
                const int wx = ((x + dx) % nr + nr) % nr, wy = ((y + dy) % nr + nr) % nr, wz = ((z + dz) % nr + nr) % nr;
                const int cx = wx / 2, cy = wy / 2, cz = wz / 2;   // bf-block of level j-1
                if (!have[j - 1].at(cx, cy, cz)) add[j - 1].at(cx, cy, cz) = 1;
              }
        }
  }
  std::fill(add[0].v.begin(), add[0].v.end(), 0);
  // 5: old boxes, then x-runs of the new blocks ordered by (z, y, x)
  out->assign(L, {});
  for (int l = 0; l < L; ++l) {
    std::vector<slh_box>& o = (*out)[l];
    o.assign(boxes + off[l], boxes + off[l + 1]);
    const int nb = add[l].n;
    for (int z = 0; z < nb; ++z)
      for (int y = 0; y < nb; ++y) {
        int x = 0;
        while (x < nb) {
          if (!add[l].at(x, y, z) || have[l].at(x, y, z)) {
            ++x;
            continue;
          }
          const int x0 = x;
          while (x < nb && add[l].at(x, y, z) && !have[l].at(x, y, z)) ++x;
          slh_box b;
          b.lo[0] = x0 * bf;
          b.lo[1] = y * bf;
          b.lo[2] = z * bf;
          b.hi[0] = x * bf - 1;
          b.hi[1] = (y + 1) * bf - 1;
          b.hi[2] = (z + 1) * bf - 1;
          o.push_back(b);
        }
      }
  }
  return SLH_OK;
}

}  // namespace slh

extern "C" slh_status slh_local_regrid_boxes(int32_t nlevels, int32_t n0, int32_t blocking_factor,
                                             const uint8_t* const* masks, const slh_box* boxes,
                                             const int32_t* nboxes, slh_box* out, int32_t cap,
                                             int32_t* out_nboxes) {
  if (nlevels < 1 || nlevels > 8 || !boxes || !nboxes || !out_nboxes)
    return slh::fail(SLH_ERR_INVALID_ARG, "local_regrid: bad arguments");
  if (blocking_factor < 2 || (blocking_factor & (blocking_factor - 1)))
    return slh::fail(SLH_ERR_INVALID_ARG, "local_regrid: blocking factor must be a power of two >= 2");
  if (n0 < blocking_factor || n0 % blocking_factor)
    return slh::fail(SLH_ERR_INVALID_ARG, "local_regrid: n0 must be a positive multiple of the blocking factor");
  std::vector<std::vector<slh_box>> res;
  slh_status st = slh::local_regrid_impl(nlevels, n0, blocking_factor, masks, boxes, nboxes, &res);
  if (st != SLH_OK) return st;
  int total = 0;
  for (int l = 0; l < nlevels; ++l) {
    out_nboxes[l] = (int32_t)res[l].size();
    total += (int)res[l].size();
  }
  if (total > cap || !out) return slh::fail(SLH_ERR_OUT_OF_RANGE, "local_regrid: %d boxes exceed capacity %d", total, cap);
  int o = 0;
  for (int l = 0; l < nlevels; ++l)
    for (const slh_box& b : res[l]) out[o++] = b;
  return SLH_OK;
}
