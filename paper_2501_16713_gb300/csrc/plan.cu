// Plan construction for the nonrigid SENSE operator (host, plan time).
//
// nrsense_plan_create validates the problem statement (stacked SENSE
// equation: P motion states sharing one image, C coils, M_j samples per
// state), evaluates the kernel polynomials and deapodization tables in FP64,
// decomposes every k-space sample position q = omega G / (2 pi) and every
// displaced voxel position q = sigma (n + d_j[n]) into first tap and fraction,
// sorts the points into 8^3 grid tiles, builds the per-tile halo lists and
// work items of the output-stationary spreading kernels, and creates the cuFFT
// plans and work buffers.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "kb_host.h"
#include <cufftXt.h>

#include "plan_internal.h"

using namespace nrs;

namespace {

// Host-side fault injection for the error paths (NRSENSE_FAULT=alloc|cufft|upload).
bool fault_requested(const char* what) {
  const char* f = std::getenv("NRSENSE_FAULT");
  return f != nullptr && std::strcmp(f, what) == 0;
}

nrsense_status dev_alloc(nrsense_plan_s* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) return NRSENSE_OK;
  if (fault_requested("alloc")) return NRSENSE_ERR_OOM;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return NRSENSE_ERR_OOM;
  }
  p->allocations.push_back(*ptr);
  p->allocation_bytes.push_back(bytes);
  p->device_bytes += (long long)bytes;
  return NRSENSE_OK;
}

// free one tracked allocation (null: no-op)
void dev_free(nrsense_plan_s* p, void* ptr) {
  if (ptr == nullptr) return;
  for (size_t i = 0; i < p->allocations.size(); ++i)
    if (p->allocations[i] == ptr) {
      cudaFree(ptr);
      p->device_bytes -= (long long)p->allocation_bytes[i];
      p->allocations.erase(p->allocations.begin() + long(i));
      p->allocation_bytes.erase(p->allocation_bytes.begin() + long(i));
      return;
    }
}

void free_pointset(nrsense_plan_s* p, PointSet* ps) {
  void* arrs[] = {ps->qs, ps->perm, ps->list, ps->items, ps->bins, ps->reduces, ps->iitems,
                  ps->clist, ps->cbins};
  for (void* a : arrs) dev_free(p, a);
  *ps = PointSet{};
}

template <typename T>
nrsense_status dev_alloc_n(nrsense_plan_s* p, T** ptr, long long n) {
  return dev_alloc(p, reinterpret_cast<void**>(ptr), size_t(n) * sizeof(T));
}

template <typename T>
nrsense_status upload(T* dst, const std::vector<T>& src, cudaStream_t s) {
  if (src.empty()) return NRSENSE_OK;
  if (fault_requested("upload")) return NRSENSE_ERR_CUDA;
  if (cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s) !=
      cudaSuccess)
    return NRSENSE_ERR_CUDA;
  // host vectors are freed by the caller after return: wait here
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

#define NRS_TRY(expr)                          \
  do {                                         \
    nrsense_status _st = (expr);               \
    if (_st != NRSENSE_OK) return _st;         \
  } while (0)

struct HostPoint {
  float f[3];
  int b[3];
  int32_t row;
};

// Decompose a position on the periodic grid: first tap index (mod G) and the
// fractional offset f = q - floor(q) of the kernel's centre cell.
inline void decompose(double q, int G, int W, int* base, float* frac) {
  const double fl = std::floor(q);
  long long b = (long long)fl - (W / 2 - 1);
  b %= G;
  if (b < 0) b += G;
  *base = int(b);
  *frac = float(q - fl);
}

inline int tile_of(int idx, int tile) { return idx / tile; }

// Sort points into tiles, build halo lists and work items, upload.
// Morton (Z-order) code of a tile, 10 bits per axis: work items in this
// order keep neighbouring tiles (which share halo data) close in time.
uint64_t morton3(const TilePlan& tp, long long tile) {
  const long long tz = tile / ((long long)tp.nt1 * tp.nt2);
  const long long rem = tile - tz * tp.nt1 * tp.nt2;
  const long long ty = rem / tp.nt2, tx = rem - ty * tp.nt2;
  uint64_t m = 0;
  for (int b = 0; b < 10; ++b) {
    m |= uint64_t((tx >> b) & 1) << (3 * b);
    m |= uint64_t((ty >> b) & 1) << (3 * b + 1);
    m |= uint64_t((tz >> b) & 1) << (3 * b + 2);
  }
  return m;
}

TilePlan make_tileplan(const Geo& g, int T) {
  TilePlan tp;
  tp.t0 = tp.t1 = tp.t2 = T;
  tp.nt0 = (g.g0 + T - 1) / T;
  tp.nt1 = (g.g1 + T - 1) / T;
  tp.nt2 = (g.g2 + T - 1) / T;
  tp.ntiles = (long long)tp.nt0 * tp.nt1 * tp.nt2;
  return tp;
}

// Mark every tile touched by a footprint of the given points.
void mark_touched_tiles(const nrsense_plan_s* p, const TilePlan& tp,
                        const std::vector<HostPoint>& pts, std::vector<char>& mask) {
  const Geo& g = p->geo;
  const int gsz[3] = {g.g0, g.g1, g.g2};
  const int tsz[3] = {tp.t0, tp.t1, tp.t2};
  for (const HostPoint& h : pts) {
    int tl[3][2], nt[3];
    for (int a = 0; a < 3; ++a) {
      nt[a] = 0;
      for (int t = 0; t < p->W; ++t) {
        int gi = h.b[a] + t;
        if (gi >= gsz[a]) gi -= gsz[a];
        const int ti = gi / tsz[a];
        if (nt[a] == 0 || tl[a][nt[a] - 1] != ti) {
          if (nt[a] < 2) tl[a][nt[a]++] = ti;
        }
      }
    }
    for (int a = 0; a < nt[0]; ++a)
      for (int b = 0; b < nt[1]; ++b)
        for (int c = 0; c < nt[2]; ++c)
          mask[((long long)tl[0][a] * tp.nt1 + tl[1][b]) * tp.nt2 + tl[2][c]] = 1;
  }
}

// write_mask: tiles that must be written even without points of this set
// (NULL = every tile).
// tp: tiles of this set; write_mask: tiles that must be written even without
// points (NULL = every tile); interp: also build interpolation work items.
nrsense_status build_pointset(nrsense_plan_s* p, std::vector<HostPoint>& pts, PointSet* ps,
                              const TilePlan& tp, const std::vector<char>* write_mask,
                              bool interp, int max_item, cudaStream_t s) {
  const Geo& g = p->geo;
  ps->tp = tp;
  const int W = p->W;
  const long long npts = (long long)pts.size();
  ps->npts = npts;
  if (npts >= (1ll << 31)) return NRSENSE_ERR_ARG;

  // primary key: tile of the first tap; secondary: cell inside the tile
  std::vector<int64_t> key(npts);
  for (long long i = 0; i < npts; ++i) {
    const HostPoint& h = pts[i];
    const long long t = ((long long)tile_of(h.b[0], tp.t0) * tp.nt1 + tile_of(h.b[1], tp.t1)) *
                            tp.nt2 + tile_of(h.b[2], tp.t2);
    const int cell = ((h.b[0] % tp.t0) * tp.t1 + (h.b[1] % tp.t1)) * tp.t2 + (h.b[2] % tp.t2);
    key[i] = t * 4096 + cell;  // cell < T^3 <= 4096
  }
  std::vector<int32_t> order(npts);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  // interpolation items: sorted ranges of points sharing a first-tap tile
  std::vector<SpreadItem> iitems;
  if (interp) {
    long long b = 0;
    while (b < npts) {
      const long long t = key[order[b]] / 4096;
      long long e = b;
      while (e < npts && key[order[e]] / 4096 == t) ++e;
      for (long long cb = b; cb < e; cb += kInterpMaxItem)
        iitems.push_back({int32_t(t), int32_t(cb), int32_t(std::min(e, cb + kInterpMaxItem)), -1});
      b = e;
    }
    std::stable_sort(iitems.begin(), iitems.end(), [&](const SpreadItem& a, const SpreadItem& b) {
      return morton3(tp, a.tile) < morton3(tp, b.tile);
    });
  }
  key.clear();
  key.shrink_to_fit();

  std::vector<float4> qs(npts);
  std::vector<int32_t> perm(npts);
  for (long long s_i = 0; s_i < npts; ++s_i) {
    const HostPoint& h = pts[order[s_i]];
    const uint32_t packed = pack_base(h.b[0], h.b[1], h.b[2]);
    float w;
    std::memcpy(&w, &packed, sizeof(w));
    qs[s_i] = make_float4(h.f[0], h.f[1], h.f[2], w);
    perm[s_i] = h.row;
  }

  // halo lists: every tile touched by a point's W^3 footprint
  const int gsz[3] = {g.g0, g.g1, g.g2};
  const int tsz[3] = {tp.t0, tp.t1, tp.t2};
  const int ntz[3] = {tp.nt0, tp.nt1, tp.nt2};
  auto touched = [&](const HostPoint& h, int a, int* out) {
    int n = 0;
    for (int t = 0; t < W; ++t) {
      int gi = h.b[a] + t;
      if (gi >= gsz[a]) gi -= gsz[a];
      const int ti = gi / tsz[a];
      bool seen = false;
      for (int k = 0; k < n; ++k) seen |= (out[k] == ti);
      if (!seen) out[n++] = ti;
    }
    (void)ntz;
    return n;
  };
  std::vector<int64_t> counts(tp.ntiles + 1, 0);
  for (long long s_i = 0; s_i < npts; ++s_i) {
    const HostPoint& h = pts[order[s_i]];
    int t0[8], t1[8], t2[8];
    const int n0 = touched(h, 0, t0), n1 = touched(h, 1, t1), n2 = touched(h, 2, t2);
    for (int a = 0; a < n0; ++a)
      for (int b = 0; b < n1; ++b)
        for (int c = 0; c < n2; ++c)
          counts[((long long)t0[a] * tp.nt1 + t1[b]) * tp.nt2 + t2[c] + 1]++;
  }
  for (long long t = 0; t < tp.ntiles; ++t) counts[t + 1] += counts[t];
  const long long list_len = counts[tp.ntiles];
  if (list_len >= (1ll << 31)) return NRSENSE_ERR_ARG;
  std::vector<int32_t> list(list_len);  // sorted indices; paired with rows below
  std::vector<int64_t> fill(counts.begin(), counts.end() - 1);
  for (long long s_i = 0; s_i < npts; ++s_i) {
    const HostPoint& h = pts[order[s_i]];
    int t0[8], t1[8], t2[8];
    const int n0 = touched(h, 0, t0), n1 = touched(h, 1, t1), n2 = touched(h, 2, t2);
    for (int a = 0; a < n0; ++a)
      for (int b = 0; b < n1; ++b)
        for (int c = 0; c < n2; ++c)
          list[fill[((long long)t0[a] * tp.nt1 + t1[b]) * tp.nt2 + t2[c]]++] = int32_t(s_i);
  }
  ps->list_len = list_len;
  // within each tile, order the points by the plane offset of their first tap
  // (axis 0) relative to the tile origin, so the spreading warp that owns a
  // plane finds its points in one contiguous range (stable: ties keep order)
  {
    const int nb = W + tp.t0;  // offsets in (-W, T)
    std::vector<int32_t> tmp;
    std::vector<int64_t> bcount(nb + 1);
    for (long long t = 0; t < tp.ntiles; ++t) {
      const long long b = counts[t], e = counts[t + 1];
      if (e - b < 2) continue;
      const int o0 = int(t / ((long long)tp.nt1 * tp.nt2)) * tp.t0;
      auto key = [&](int32_t si) {
        int r = pts[order[si]].b[0] - o0;
        if (r < 0) r += g.g0;
        if (r >= tp.t0) r -= g.g0;
        return r + W - 1;
      };
      std::fill(bcount.begin(), bcount.end(), 0);
      for (long long i = b; i < e; ++i) bcount[key(list[i]) + 1]++;
      for (int k = 0; k < nb; ++k) bcount[k + 1] += bcount[k];
      tmp.assign(list.begin() + b, list.begin() + e);
      for (int32_t si : tmp) list[b + bcount[key(si)]++] = si;
    }
  }

  // work items: occupied tiles, plus empty tiles in write_mask (they write
  // zeros); heavy tiles split
  std::vector<SpreadItem> items;
  std::vector<ReduceItem> reds;
  int slots = 0, occupied = 0;
  for (long long t = 0; t < tp.ntiles; ++t) {
    const long long b = counts[t], e = counts[t + 1];
    const long long L = e - b;
    if (L > 0) occupied++;
    if (L == 0 && write_mask != nullptr && !(*write_mask)[t]) continue;
    if (L <= max_item) {
      items.push_back({int32_t(t), int32_t(b), int32_t(e), -1});
    } else {
      // deal the (r0-sorted) entries round-robin into chunks, so every chunk
      // spans all planes of the tile and keeps the r0 order
      const int nchunk = int((L + max_item - 1) / max_item);
      std::vector<int32_t> seg(list.begin() + b, list.begin() + e);
      long long w = b;
      ReduceItem r{int32_t(t), slots, nchunk, 0};
      for (int k = 0; k < nchunk; ++k) {
        const long long cb = w;
        for (long long i = k; i < L; i += nchunk) list[w++] = seg[i];
        items.push_back({int32_t(t), int32_t(cb), int32_t(w), slots + k});
      }
      slots += nchunk;
      reds.push_back(r);
    }
  }
  // Morton order of tiles (chunks of a tile stay adjacent)
  std::stable_sort(items.begin(), items.end(), [&](const SpreadItem& a, const SpreadItem& b) {
    return morton3(tp, a.tile) < morton3(tp, b.tile);
  });
  ps->n_items = int(items.size());
  ps->n_reduces = int(reds.size());
  ps->n_slots = slots;
  ps->n_occupied = occupied;
  ps->n_iitems = int(iitems.size());
  // per item: first entry of each first-tap plane offset bin (list sorted by
  // r0 within every tile, so within every item)
  const int nb = W + tp.t0 + 1;
  std::vector<int32_t> bins((size_t)items.size() * nb);
  for (size_t k = 0; k < items.size(); ++k) {
    const SpreadItem& itm = items[k];
    const int o0 = int(itm.tile / ((long long)tp.nt1 * tp.nt2)) * tp.t0;
    int32_t* bk = bins.data() + k * nb;
    int e = itm.begin;
    for (int bb = 0; bb < nb - 1; ++bb) {
      // advance past entries with r0 + W - 1 < bb
      while (e < itm.end) {
        int r = pts[order[list[e]]].b[0] - o0;
        if (r < 0) r += g.g0;
        if (r >= tp.t0) r -= g.g0;
        if (r + W - 1 >= bb) break;
        ++e;
      }
      bk[bb] = e - itm.begin;
    }
    bk[nb - 1] = itm.end - itm.begin;
  }
  // class-ordered copy for the tensor-core spread over 4^3 sub-blocks (8^3
  // tiles, W = 4): along each axis the first-tap offset r in [-3, 7] puts a
  // footprint in the low half of the tile only (r <= 0), in both halves
  // (1 <= r <= 3) or in the high half only (r >= 4); the entries of every item
  // are ordered by class 9 c0 + 3 c1 + c2 (stable), with 28 offsets per item
  const bool cube = W == 4 && tp.t0 == 8 && tp.t1 == 8 && tp.t2 == 8;
  std::vector<int2> clist2;
  std::vector<int32_t> cbins;
  if (cube) {
    clist2.resize(list_len);
    cbins.assign(items.size() * kCubeBins, 0);
    std::vector<int32_t> cls;
    for (size_t k = 0; k < items.size(); ++k) {
      const SpreadItem& itm = items[k];
      const long long t = itm.tile;
      const int o[3] = {int(t / ((long long)tp.nt1 * tp.nt2)) * 8, int((t / tp.nt2) % tp.nt1) * 8,
                        int(t % tp.nt2) * 8};
      const int n = itm.end - itm.begin;
      cls.resize(n);
      int32_t* cb = cbins.data() + k * kCubeBins;
      for (int i = 0; i < n; ++i) {
        const HostPoint& h = pts[order[list[itm.begin + i]]];
        int c = 0;
        for (int a = 0; a < 3; ++a) {
          int r = h.b[a] - o[a];
          if (r < 0) r += gsz[a];
          if (r >= 8) r -= gsz[a];
          c = 3 * c + (r <= 0 ? 0 : r < 4 ? 1 : 2);
        }
        cls[i] = c;
        cb[c + 1]++;
      }
      for (int c = 0; c < kCubeBins - 1; ++c) cb[c + 1] += cb[c];
      std::vector<int32_t> at(cb, cb + kCubeBins - 1);
      for (int i = 0; i < n; ++i) {
        const int32_t si = list[itm.begin + i];
        clist2[itm.begin + at[cls[i]]++] = make_int2(si, perm[si]);
      }
    }
  }
  std::vector<int2> list2(list_len);
  for (long long i = 0; i < list_len; ++i) list2[i] = make_int2(list[i], perm[list[i]]);
  std::vector<int32_t>().swap(list);

  NRS_TRY(dev_alloc_n(p, &ps->qs, std::max<long long>(npts, 1)));
  NRS_TRY(dev_alloc_n(p, &ps->perm, std::max<long long>(npts, 1)));
  NRS_TRY(dev_alloc_n(p, &ps->list, std::max<long long>(list_len, 1)));
  NRS_TRY(dev_alloc_n(p, &ps->items, std::max<long long>((long long)items.size(), 1)));
  NRS_TRY(dev_alloc_n(p, &ps->bins, std::max<long long>((long long)bins.size(), 1)));
  NRS_TRY(dev_alloc_n(p, &ps->reduces, std::max<long long>((long long)reds.size(), 1)));
  NRS_TRY(dev_alloc_n(p, &ps->iitems, std::max<long long>((long long)iitems.size(), 1)));
  NRS_TRY(upload(ps->qs, qs, s));
  NRS_TRY(upload(ps->perm, perm, s));
  NRS_TRY(upload(ps->list, list2, s));
  NRS_TRY(upload(ps->items, items, s));
  NRS_TRY(upload(ps->bins, bins, s));
  NRS_TRY(upload(ps->reduces, reds, s));
  NRS_TRY(upload(ps->iitems, iitems, s));
  if (cube) {
    NRS_TRY(dev_alloc_n(p, &ps->clist, std::max<long long>(list_len, 1)));
    NRS_TRY(dev_alloc_n(p, &ps->cbins, std::max<long long>((long long)cbins.size(), 1)));
    NRS_TRY(upload(ps->clist, clist2, s));
    NRS_TRY(upload(ps->cbins, cbins, s));
  }
  return NRSENSE_OK;
}

// Image-space points sorted by the 8^3 home tile of their first tap, then by
// cell (the order of the home-tile spread, spread_home.cu), with the first
// sorted index of every home tile, and the super-tile scratch.
nrsense_status build_home_set(nrsense_plan_s* p, const std::vector<HostPoint>& pts,
                              cudaStream_t s) {
  const Geo& g = p->geo;
  HomeSet& hs = p->ihome;
  hs.nt0 = (g.g0 + 7) / 8;
  hs.nt1 = (g.g1 + 7) / 8;
  hs.nt2 = (g.g2 + 7) / 8;
  hs.ns0 = (g.g0 + 15) / 16;
  hs.ns1 = (g.g1 + 15) / 16;
  hs.ns2 = (g.g2 + 15) / 16;
  const long long ntl = (long long)hs.nt0 * hs.nt1 * hs.nt2;
  const long long npts = (long long)pts.size();
  // (key << 32 | index): sorting by it is stable in the input order
  std::vector<uint64_t> ko(npts);
  std::vector<int32_t> tstart(ntl + 1, 0);
  for (long long i = 0; i < npts; ++i) {
    const HostPoint& h = pts[i];
    const long long t = ((long long)(h.b[0] >> 3) * hs.nt1 + (h.b[1] >> 3)) * hs.nt2 + (h.b[2] >> 3);
    const int cell = (((h.b[0] & 7) * 8) + (h.b[1] & 7)) * 8 + (h.b[2] & 7);
    ko[i] = (uint64_t(t * 512 + cell) << 32) | uint64_t(i);
    tstart[t + 1]++;
  }
  std::sort(ko.begin(), ko.end());
  for (long long t = 0; t < ntl; ++t) tstart[t + 1] += tstart[t];
  std::vector<float4> qs(std::max<long long>(npts, 1));
  std::vector<int32_t> perm(std::max<long long>(npts, 1));
  for (long long k = 0; k < npts; ++k) {
    const HostPoint& h = pts[ko[k] & 0xffffffffu];
    const uint32_t packed = pack_base(h.b[0], h.b[1], h.b[2]);
    float w;
    std::memcpy(&w, &packed, sizeof(w));
    qs[k] = make_float4(h.f[0], h.f[1], h.f[2], w);
    perm[k] = h.row;
  }
  std::vector<uint64_t>().swap(ko);
  float4* dq = nullptr;
  int32_t *dp = nullptr, *dt = nullptr;
  NRS_TRY(dev_alloc_n(p, &dq, (long long)qs.size()));
  NRS_TRY(dev_alloc_n(p, &dp, (long long)perm.size()));
  NRS_TRY(dev_alloc_n(p, &dt, ntl + 1));
  NRS_TRY(upload(dq, qs, s));
  NRS_TRY(upload(dp, perm, s));
  NRS_TRY(upload(dt, tstart, s));
  hs.qs = dq;
  hs.perm = dp;
  hs.tstart = dt;
  // per axis and coordinate: the super-tiles whose 3-point-padded extents
  // cover it (directly or wrapped around the periodic grid), increasing
  const int gsz[3] = {g.g0, g.g1, g.g2}, nsz[3] = {hs.ns0, hs.ns1, hs.ns2};
  const int4** cov[3] = {&hs.cover0, &hs.cover1, &hs.cover2};
  for (int a = 0; a < 3; ++a) {
    std::vector<int4> tab(gsz[a]);
    for (int x = 0; x < gsz[a]; ++x) {
      int e[3] = {0, 0, 0}, n = 0;
      for (int c = 0; c < nsz[a]; ++c) {
        const int o = 16 * c, ext = std::min(16, gsz[a] - o);
        for (int u : {x, x + gsz[a]})
          if (u >= o && u < o + ext + 3) {
            if (n == 3) return NRSENSE_ERR_ARG;  // cannot happen for grids >= 11 points
            e[n++] = c * 32 + (u - o);
          }
      }
      tab[x] = make_int4(n, e[0], e[1], e[2]);
    }
    int4* dtab = nullptr;
    NRS_TRY(dev_alloc_n(p, &dtab, (long long)tab.size()));
    NRS_TRY(upload(dtab, tab, s));
    if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
    *cov[a] = dtab;
  }
  NRS_TRY(dev_alloc_n(p, &p->home_scratch, home_scratch_elems(hs)));
  if (configure_home_kernels() != cudaSuccess) return NRSENSE_ERR_CUDA;
  p->home_ok = true;
  // host vectors are freed on return: wait for the uploads
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

// scratch for split tiles: slots x coil chunks x tile x chunk coils (grown,
// never shrunk)
nrsense_status ensure_scratch(nrsense_plan_s* p) {
  long long need = 0;
  auto tile_pts = [](const PointSet& ps) {
    return (long long)ps.tp.t0 * ps.tp.t1 * ps.tp.t2;
  };
  if (!p->identity_warp) need = std::max(need, (long long)p->ipts.n_slots * tile_pts(p->ipts));
  if (p->C > 0) {
    const int cc = spread_coil_chunk(p->C);
    const int chunks = (p->C + cc - 1) / cc;
    for (int j0 = 0; j0 < p->P; j0 += p->phase_chunk) {
      long long slots = 0;
      for (int j = j0; j < std::min(p->P, j0 + p->phase_chunk); ++j) slots += p->kpts[j].n_slots;
      need = std::max(need, slots * chunks * tile_pts(p->kpts[j0]) * cc);
    }
  }
  if (need <= p->scratch_elems) return NRSENSE_OK;
  dev_free(p, p->b_scratch);
  p->b_scratch = nullptr;
  p->scratch_elems = 0;
  NRS_TRY(dev_alloc_n(p, &p->b_scratch, need));
  p->scratch_elems = need;
  return NRSENSE_OK;
}

nrsense_status cufft_check(cufftResult r) {
  return r == CUFFT_SUCCESS ? NRSENSE_OK : NRSENSE_ERR_CUFFT;
}

nrsense_status create_impl(nrsense_plan_s* p, const nrsense_desc* desc, const int64_t* n_samples,
                           const float* coords, const float* disp, const nrsense_c64* smaps,
                           cudaStream_t s) {
  const nrsense_desc& d = *desc;
  for (int a = 0; a < 3; ++a)
    if (d.n[a] < 4 || (d.n[a] & 1)) return NRSENSE_ERR_ARG;
  // oversampled grid: osf * n, or given per axis (a rational sigma = G / n)
  const bool explicit_grid = d.grid[0] > 0 && d.grid[1] > 0 && d.grid[2] > 0;
  if (!explicit_grid && (d.grid[0] != 0 || d.grid[1] != 0 || d.grid[2] != 0)) return NRSENSE_ERR_ARG;
  int gsize[3];
  if (explicit_grid) {
    for (int a = 0; a < 3; ++a) {
      gsize[a] = d.grid[a];
      if (4 * gsize[a] < 5 * d.n[a] || gsize[a] > 4 * d.n[a]) return NRSENSE_ERR_ARG;
      if ((long long)gsize[a] * d.n[0] != (long long)gsize[0] * d.n[a]) return NRSENSE_ERR_ARG;
    }
  } else {
    if (d.osf < 2 || d.osf > 4) return NRSENSE_ERR_ARG;
    for (int a = 0; a < 3; ++a) gsize[a] = d.osf * d.n[a];
  }
  if (d.kb_width != 4 && d.kb_width != 6) return NRSENSE_ERR_ARG;
  if (d.n_phases < 1 || d.n_coils < 0) return NRSENSE_ERR_ARG;
  if (d.precision != NRSENSE_FP32 && d.precision != NRSENSE_BF16_STORE &&
      d.precision != NRSENSE_FP32_COMPENSATED)
    return NRSENSE_ERR_ARG;
  if (d.precision == NRSENSE_FP32_COMPENSATED && d.kb_width != 4) return NRSENSE_ERR_ARG;
  if (d.precision == NRSENSE_BF16_STORE)  // cuFFT's BF16 transforms: power-of-two sizes
    for (int a = 0; a < 3; ++a) {
      const int ga = gsize[a];
      if (ga & (ga - 1)) return NRSENSE_ERR_ARG;
    }
  if (!(d.kb_beta >= 0.0) || !std::isfinite(d.kb_beta)) return NRSENSE_ERR_ARG;
  p->desc = d;
  p->identity_warp = (d.flags & NRSENSE_IDENTITY_WARP) != 0;
  p->grid_bf16 = d.precision == NRSENSE_BF16_STORE;
  p->comp_spread = d.precision == NRSENSE_FP32_COMPENSATED;
  p->P = d.n_phases;
  p->C = d.n_coils;
  p->W = d.kb_width;
  Geo& g = p->geo;
  g.n0 = d.n[0]; g.n1 = d.n[1]; g.n2 = d.n[2];
  g.g0 = gsize[0]; g.g1 = gsize[1]; g.g2 = gsize[2];
  // integer sigma (0 when sigma = G / n is not an integer)
  g.osf = (g.g0 % g.n0 == 0) ? g.g0 / g.n0 : 0;
  const double sigma = double(g.g0) / double(g.n0);
  if (g.g0 > 1024 || g.g1 > 1024 || g.g2 > 1024) return NRSENSE_ERR_ARG;  // 10-bit packed taps
  // a tile and a kernel footprint must not wrap onto each other
  const int gmin = kSpreadTile + d.kb_width - 1;
  if (g.g0 < gmin || g.g1 < gmin || g.g2 < gmin) return NRSENSE_ERR_ARG;
  g.nvox = (long long)g.n0 * g.n1 * g.n2;
  g.ngrid = (long long)g.g0 * g.g1 * g.g2;
  if ((long long)p->P * g.nvox >= (1ll << 31)) return NRSENSE_ERR_ARG;
  if (!p->identity_warp && disp == nullptr) return NRSENSE_ERR_ARG;
  if (p->C > 0 && (coords == nullptr || smaps == nullptr || n_samples == nullptr))
    return NRSENSE_ERR_ARG;
  p->beta = d.kb_beta > 0 ? d.kb_beta : beatty_beta(p->W, sigma);
  if (!(p->beta > 0)) return NRSENSE_ERR_ARG;
  p->poly_err = fit_kernel_polys(p->W, p->beta, &p->kc);

  if (configure_kernels() != cudaSuccess) return NRSENSE_ERR_CUDA;
  const TilePlan ktiles = make_tileplan(g, kSpreadTile);
  const TilePlan itiles =
      make_tileplan(g, spread_tile_edge(p->W, 1, std::min(g.g0, std::min(g.g1, g.g2))));
  p->ktiles = ktiles;
  p->itiles = itiles;

  // deapodization: 1/C(m/G) for m in [-N/2, N/2), per axis
  {
    std::vector<float> tab;
    const int ns[3] = {g.n0, g.n1, g.n2}, gs[3] = {g.g0, g.g1, g.g2};
    for (int a = 0; a < 3; ++a)
      for (int m = -ns[a] / 2; m < ns[a] / 2; ++m)
        tab.push_back(float(1.0 / kb_kernel_ft(double(m) / gs[a], p->W, p->beta)));
    NRS_TRY(dev_alloc_n(p, &p->deapod, (long long)tab.size()));
    NRS_TRY(upload(p->deapod, tab, s));
  }
  NRS_TRY(dev_alloc_n(p, &p->d_status, 1));
  if (cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s) != cudaSuccess) return NRSENSE_ERR_CUDA;

  // displacements: copy, validate, and build the image-space point set
  if (!p->identity_warp) {
    const long long nd = (long long)p->P * 3 * g.nvox;
    NRS_TRY(dev_alloc_n(p, &p->disp, nd));
    if (cudaMemcpyAsync(p->disp, disp, size_t(nd) * sizeof(float), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
      return NRSENSE_ERR_CUDA;
    std::vector<float> hd(nd);
    if (cudaMemcpyAsync(hd.data(), disp, size_t(nd) * sizeof(float), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    for (long long i = 0; i < nd; ++i)
      if (!std::isfinite(hd[i]) || std::fabs(hd[i]) > 1e6f) return NRSENSE_ERR_ARG;
    std::vector<HostPoint> pts((size_t)(p->P * g.nvox));
    const int gs[3] = {g.g0, g.g1, g.g2};
    for (int j = 0; j < p->P; ++j) {
      const float* dj = hd.data() + (long long)j * 3 * g.nvox;
      for (long long v = 0; v < g.nvox; ++v) {
        const int i2 = int(v % g.n2);
        const int i1 = int((v / g.n2) % g.n1);
        const int i0 = int(v / ((long long)g.n1 * g.n2));
        const int ii[3] = {i0, i1, i2};
        HostPoint& h = pts[(size_t)(j * g.nvox + v)];
        for (int a = 0; a < 3; ++a) {
          // q = sigma * (n + d) = sigma*n + sigma*d in FP64 (sigma*n exact)
          const double q = sigma * double(ii[a]) + sigma * double(dj[a * g.nvox + v]);
          decompose(q, gs[a], p->W, &h.b[a], &h.f[a]);
        }
        h.row = int32_t(j * g.nvox + v);
      }
    }
    NRS_TRY(build_pointset(p, pts, &p->ipts, itiles, nullptr, /*interp=*/false,
                           kSpreadMaxItemImage, s));
    // home-tile spread (W = 4, plain FP32 accumulation); the default where built
    if (p->W == 4 && !p->comp_spread) {
      NRS_TRY(build_home_set(p, pts, s));
      p->spread_image_variant = kSpreadHome;
      p->interp_home = true;
    }
  }

  // coils and k-space
  if (p->C > 0) {
    p->M.assign(n_samples, n_samples + p->P);
    p->off.resize(p->P);
    long long tot = 0;
    for (int j = 0; j < p->P; ++j) {
      if (p->M[j] < 0 || p->M[j] >= (1ll << 31)) return NRSENSE_ERR_ARG;
      p->off[j] = tot;
      tot += p->M[j];
    }
    p->Mtot = tot;
    const long long nm = g.nvox * p->C;
    NRS_TRY(dev_alloc_n(p, &p->smaps, nm));
    if (cudaMemcpyAsync(p->smaps, smaps, size_t(nm) * sizeof(nrsense_c64), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;

    std::vector<float> hc(size_t(3 * tot));
    if (tot > 0) {
      if (cudaMemcpyAsync(hc.data(), coords, size_t(3 * tot) * sizeof(float),
                          cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        return NRSENSE_ERR_CUDA;
    }
    p->kpts.resize(p->P);
    const int gs[3] = {g.g0, g.g1, g.g2};
    std::vector<std::vector<HostPoint>> all((size_t)p->P);
    for (int j = 0; j < p->P; ++j) {
      std::vector<HostPoint>& pts = all[(size_t)j];
      pts.resize((size_t)p->M[j]);
      for (long long i = 0; i < p->M[j]; ++i) {
        HostPoint& h = pts[(size_t)i];
        for (int a = 0; a < 3; ++a) {
          const float om = hc[size_t(3 * (p->off[j] + i) + a)];
          if (!std::isfinite(om)) return NRSENSE_ERR_ARG;
          // q = omega G / (2 pi) in FP64; periodic, so any finite omega wraps
          const double q = double(om) * double(gs[a]) / (2.0 * M_PI);
          decompose(q, gs[a], p->W, &h.b[a], &h.f[a]);
        }
        h.row = int32_t(i);
      }
    }
    // all phases share one spread target: each phase writes every tile that
    // any phase occupies (zeros where it has no points), the rest stay zero
    std::vector<char> uni((size_t)ktiles.ntiles, 0);
    for (int j = 0; j < p->P; ++j) mark_touched_tiles(p, ktiles, all[(size_t)j], uni);
    long long nuni = 0;
    for (char u : uni) nuni += u != 0;
    p->kuni_fraction = double(nuni) / double(uni.size());
    // per (y, x) tile column, a bit per z tile of the union: the pruned
    // transforms store (forward) and load (adjoint) only those tiles
    if (ktiles.nt0 <= 32) {
      std::vector<uint32_t> cm((size_t)ktiles.nt1 * ktiles.nt2, 0u);
      long long ncol = 0;
      for (long long t = 0; t < ktiles.ntiles; ++t)
        if (uni[(size_t)t]) {
          const long long col = t % ((long long)ktiles.nt1 * ktiles.nt2);
          cm[(size_t)col] |= 1u << int(t / ((long long)ktiles.nt1 * ktiles.nt2));
        }
      for (uint32_t v : cm) ncol += v != 0u;
      p->kcol_fraction = double(ncol) / double(cm.size());
      NRS_TRY(dev_alloc_n(p, &p->kcolmask, (long long)cm.size()));
      NRS_TRY(upload(p->kcolmask, cm, s));
    }
    for (int j = 0; j < p->P; ++j) {
      NRS_TRY(build_pointset(p, all[(size_t)j], &p->kpts[j], ktiles, &uni, /*interp=*/true,
                             p->spread_max_item, s));
      std::vector<HostPoint>().swap(all[(size_t)j]);
    }
    p->kunion.swap(uni);
  }

  // cuFFT plans
  if (fault_requested("cufft")) return NRSENSE_ERR_CUFFT;
  if (!p->identity_warp) {
    NRS_TRY(cufft_check(cufftPlan3d(&p->fft_n, g.n0, g.n1, g.n2, CUFFT_C2C)));
    p->have_fft_n = true;
    NRS_TRY(cufft_check(cufftPlan3d(&p->fft_g, g.g0, g.g1, g.g2, CUFFT_C2C)));
    p->have_fft_g = true;
  }
  if (p->C > 0) {
    // phases per launch: as many as half of the free memory allows (four
    // coil-grid buffers per phase plus about one for cuFFT's work area)
    const long long elem = p->grid_bf16 ? 4 : 8;  // bytes per stored complex value
    const long long per_phase = 5LL * p->C * g.ngrid * elem;
    int pc = d.phase_chunk;
    if (pc <= 0) {
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return NRSENSE_ERR_CUDA;
      pc = int(std::max<long long>(1, (long long)(free_b / 2) / per_phase));
    }
    pc = std::max(1, std::min(pc, std::min(p->P, kMaxChunkPhases)));
    p->phase_chunk = pc;
    // pruned coil-grid transforms (FP32 C2C or BF16 through cufftXt)
    const long long plane = (long long)g.g1 * g.g2;
    long long n2[2] = {g.g1, g.g2};
    long long nz[1] = {g.g0};
    auto make = [&](cufftHandle* h, int rank, long long* n, long long* emb, long long stride,
                    long long dist, long long batch) -> nrsense_status {
      if (cufftCreate(h) != CUFFT_SUCCESS) return NRSENSE_ERR_CUFFT;
      size_t work = 0;
      const cufftResult r =
          p->grid_bf16
              ? cufftXtMakePlanMany(*h, rank, n, emb, stride, dist, CUDA_C_16BF, emb, stride, dist,
                                    CUDA_C_16BF, batch, &work, CUDA_C_16BF)
              : cufftMakePlanMany64(*h, rank, n, emb, stride, dist, emb, stride, dist, CUFFT_C2C,
                                    batch, &work);
      if (r != CUFFT_SUCCESS) {
        cufftDestroy(*h);
        return NRSENSE_ERR_CUFFT;
      }
      return NRSENSE_OK;
    };
    NRS_TRY(make(&p->fft_p2, 2, n2, n2, 1, plane, g.n0));
    nrsense_status st2 = make(&p->fft_p2h, 2, n2, n2, 1, plane, g.n0 / 2);
    if (st2 != NRSENSE_OK) {
      cufftDestroy(p->fft_p2);
      return st2;
    }
    st2 = make(&p->fft_z, 1, nz, nz, plane, 1, plane);
    if (st2 != NRSENSE_OK) {
      cufftDestroy(p->fft_p2);
      cufftDestroy(p->fft_p2h);
      return st2;
    }
    p->have_gc = true;
  }

  // work buffers
  NRS_TRY(dev_alloc_n(p, &p->b_m, (long long)p->P * g.nvox));
  NRS_TRY(dev_alloc_n(p, &p->b_tmp, g.nvox));
  if (!p->identity_warp) {
    NRS_TRY(dev_alloc_n(p, &p->b_xhat, g.nvox));
    NRS_TRY(dev_alloc_n(p, &p->b_upad, g.ngrid));
    NRS_TRY(dev_alloc_n(p, &p->b_ugrid, g.ngrid));
    if (cudaMemsetAsync(p->b_upad, 0, size_t(g.ngrid) * sizeof(nrsense_c64), s) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    // the pruned image-space passes: their T1 and T2 (6 N^3 values) fit in b_upad (8 N^3)
    p->image_fft_ok = pruned_image_fft_supported(g) && !p->comp_spread;
    p->image_fft_pruned = p->image_fft_ok;
  }
  if (p->C > 0) {
    const size_t cgb = size_t(g.ngrid) * p->C * p->phase_chunk * (p->grid_bf16 ? 4 : 8);
    NRS_TRY(dev_alloc(p, &p->b_xpad, cgb));
    NRS_TRY(dev_alloc(p, &p->b_xwork, cgb));
    NRS_TRY(dev_alloc(p, &p->b_xspread, cgb));
    NRS_TRY(dev_alloc(p, &p->b_xmid, cgb));
    if (cudaMemsetAsync(p->b_xmid, 0, cgb, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
    // own pruned transforms where supported (chosen by default; the autotuner
    // times both paths)
    p->fft_pruned_ok = pruned_fft_supported(g, p->C, p->grid_bf16) && init_pruned_fft() == cudaSuccess;
    p->fft_pruned = p->fft_pruned_ok;
    // tensor maps of the interpolation input (TMA-staged halos, W = 4)
    const long long slots = (long long)p->C * p->phase_chunk;
    // a test-only limit on the halo wait (0 makes every TMA-staged CTA time out)
    if (const char* lim = std::getenv("NRSENSE_TMA_POLL_LIMIT")) p->tma_poll_limit = std::atoll(lim);
    p->tma_ok = p->W == 4 &&
                make_grid_tensor_map(&p->tmap_xwork4, p->b_xwork, g, slots, p->grid_bf16, 4) &&
                make_grid_tensor_map(&p->tmap_xwork8, p->b_xwork, g, slots, p->grid_bf16, 8) &&
                make_grid_tensor_map(&p->tmap_xwork2, p->b_xwork, g, slots, p->grid_bf16, 2);
    // empty tiles of the spread target are never written: zero them once
    if (cudaMemsetAsync(p->b_xspread, 0, cgb, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
    NRS_TRY(dev_alloc_n(p, &p->b_y, std::max<long long>(p->Mtot * p->C, 1)));
    if (cudaMemsetAsync(p->b_xpad, 0, cgb, s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  }
  NRS_TRY(ensure_scratch(p));
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

void release(nrsense_plan_s* p) {
  cg_release(p);
  fista_release(p);
  motion_release(p);
  for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
  p->prof_events.clear();
  if (p->have_fft_n) cufftDestroy(p->fft_n);
  if (p->have_fft_g) cufftDestroy(p->fft_g);
  if (p->have_gc) {
    cufftDestroy(p->fft_p2);
    cufftDestroy(p->fft_p2h);
    cufftDestroy(p->fft_z);
    p->have_gc = false;
  }
  for (void* a : p->allocations) cudaFree(a);
  p->allocations.clear();
  p->allocation_bytes.clear();
}

}  // namespace

namespace nrs {

nrsense_status retile_kspace(nrsense_plan_s* p, int max_item, cudaStream_t s) {
  p->epoch += 1;  // point-set buffers are rebuilt
  if (max_item < 64 || max_item > (1 << 16)) return NRSENSE_ERR_ARG;
  if (p->C == 0 || max_item == p->spread_max_item) {
    p->spread_max_item = p->C == 0 ? p->spread_max_item : max_item;
    return NRSENSE_OK;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  for (int j = 0; j < p->P; ++j) {
    PointSet& ps = p->kpts[j];
    // the sorted points, back to host records (their order is kept by the
    // stable sort of build_pointset)
    std::vector<float4> qs((size_t)ps.npts);
    std::vector<int32_t> perm((size_t)ps.npts);
    if (ps.npts > 0 &&
        (cudaMemcpyAsync(qs.data(), ps.qs, qs.size() * sizeof(float4), cudaMemcpyDeviceToHost,
                         s) != cudaSuccess ||
         cudaMemcpyAsync(perm.data(), ps.perm, perm.size() * sizeof(int32_t),
                         cudaMemcpyDeviceToHost, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
      return NRSENSE_ERR_CUDA;
    std::vector<HostPoint> pts((size_t)ps.npts);
    for (size_t i = 0; i < pts.size(); ++i) {
      uint32_t packed;
      std::memcpy(&packed, &qs[i].w, sizeof(packed));
      unpack_base(packed, pts[i].b[0], pts[i].b[1], pts[i].b[2]);
      pts[i].f[0] = qs[i].x;
      pts[i].f[1] = qs[i].y;
      pts[i].f[2] = qs[i].z;
      pts[i].row = perm[i];
    }
    PointSet fresh;
    NRS_TRY(build_pointset(p, pts, &fresh, ps.tp, &p->kunion, /*interp=*/true, max_item, s));
    free_pointset(p, &ps);
    ps = fresh;
  }
  p->spread_max_item = max_item;
  NRS_TRY(ensure_scratch(p));
  return cudaStreamSynchronize(s) == cudaSuccess ? NRSENSE_OK : NRSENSE_ERR_CUDA;
}

}  // namespace nrs

extern "C" {

nrsense_status nrsense_plan_create(const nrsense_desc* desc, const int64_t* n_samples_host,
                                   const float* coords_dev, const float* disp_dev,
                                   const nrsense_c64* smaps_dev, void* stream,
                                   nrsense_plan_t* out) {
  if (desc == nullptr || out == nullptr) return NRSENSE_ERR_ARG;
  *out = nullptr;
  auto* p = new (std::nothrow) nrsense_plan_s();
  if (p == nullptr) return NRSENSE_ERR_OOM;
  nrsense_status st;
  try {
    st = create_impl(p, desc, n_samples_host, coords_dev, disp_dev, smaps_dev,
                     static_cast<cudaStream_t>(stream));
  } catch (const std::bad_alloc&) {
    st = NRSENSE_ERR_OOM;
  }
  if (st != NRSENSE_OK) {
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    release(p);
    delete p;
    return st;
  }
  *out = p;
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_destroy(nrsense_plan_t plan) {
  if (plan == nullptr) return NRSENSE_OK;
  cudaDeviceSynchronize();
  release(plan);
  delete plan;
  return NRSENSE_OK;
}

nrsense_status nrsense_plan_info(nrsense_plan_t p, nrsense_info* out) {
  if (p == nullptr || out == nullptr) return NRSENSE_ERR_ARG;
  std::memset(out, 0, sizeof(*out));
  out->grid[0] = p->geo.g0;
  out->grid[1] = p->geo.g1;
  out->grid[2] = p->geo.g2;
  out->kb_beta = p->beta;
  out->kernel_poly_err = p->poly_err;
  out->total_samples = p->Mtot;
  const TilePlan& ktp = p->kpts.empty() ? p->ipts.tp : p->kpts[0].tp;
  out->tile[0] = ktp.t0;
  out->tile[1] = ktp.t1;
  out->tile[2] = ktp.t2;
  out->n_tiles = ktp.ntiles;
  long long occ = 0, items = 0, split = 0;
  for (const auto& k : p->kpts) {
    occ += k.n_occupied;
    items += k.n_items;
    split += k.n_reduces;
  }
  out->occupied_fraction =
      p->kpts.empty() ? 0.0 : double(occ) / (double(ktp.ntiles) * double(p->kpts.size()));
  out->spread_items = items;
  out->split_tiles = split;
  out->device_bytes = p->device_bytes;
  out->phase_chunk = p->phase_chunk;
  out->union_fraction = p->kuni_fraction;
  out->union_columns = p->kcol_fraction;
  return NRSENSE_OK;
}

nrsense_status nrsense_profile_start(nrsense_plan_t p, int32_t max_launches) {
  if (p == nullptr || max_launches < 0 || max_launches > (1 << 20)) return NRSENSE_ERR_ARG;
  while (p->prof_events.size() < size_t(2 * max_launches)) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return NRSENSE_ERR_CUDA;
    p->prof_events.push_back(e);
  }
  p->prof_stage.clear();
  p->prof_on = true;
  p->launches_at_start = p->launches;
  return NRSENSE_OK;
}

nrsense_status nrsense_profile_stop(nrsense_plan_t p, double* ms, int64_t* count,
                                    int64_t* own_kernels) {
  if (p == nullptr) return NRSENSE_ERR_ARG;
  p->prof_on = false;
  if (cudaDeviceSynchronize() != cudaSuccess) return NRSENSE_ERR_CUDA;
  if (ms) for (int i = 0; i < NRSENSE_NUM_STAGES; ++i) ms[i] = 0.0;
  if (count) for (int i = 0; i < NRSENSE_NUM_STAGES; ++i) count[i] = 0;
  for (size_t k = 0; k < p->prof_stage.size(); ++k) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p->prof_events[2 * k], p->prof_events[2 * k + 1]) != cudaSuccess)
      return NRSENSE_ERR_CUDA;
    const int st = p->prof_stage[k];
    if (ms) ms[st] += double(t);
    if (count) count[st] += 1;
  }
  if (own_kernels) *own_kernels = p->launches - p->launches_at_start;
  p->prof_stage.clear();
  return NRSENSE_OK;
}

const char* nrsense_stage_name(int32_t st) {
  static const char* names[NRSENSE_NUM_STAGES] = {
      "fft_n", "fft_g", "fft_gc", "deapod_pad", "interp_image", "spread_image", "crop_deapod",
      "coil_fanout_pad", "interp_kspace", "spread_kspace", "crop_coilsum", "vector", "solver",
      "cnn", "fista", "fft_pruned"};
  return (st >= 0 && st < NRSENSE_NUM_STAGES) ? names[st] : "unknown";
}

const char* nrsense_status_string(nrsense_status s) {
  switch (s) {
    case NRSENSE_OK: return "ok";
    case NRSENSE_ERR_ARG: return "invalid argument";
    case NRSENSE_ERR_OOM: return "out of memory";
    case NRSENSE_ERR_CUFFT: return "cuFFT failure";
    case NRSENSE_ERR_CUDA: return "CUDA runtime failure";
    case NRSENSE_ERR_BREAKDOWN: return "CG breakdown";
    case NRSENSE_ERR_NOT_CONVERGED: return "CG not converged";
    case NRSENSE_ERR_TIMEOUT: return "device wait timed out";
    case NRSENSE_ERR_STATE: return "call not valid for this plan";
    default: return "unknown status";
  }
}

nrsense_status nrsense_device_status(nrsense_plan_t p, int32_t clear, int32_t* out_host,
                                     void* stream) {
  if (p == nullptr || out_host == nullptr) return NRSENSE_ERR_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(out_host, p->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (clear && cudaMemsetAsync(p->d_status, 0, sizeof(int32_t), s) != cudaSuccess)
    return NRSENSE_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return NRSENSE_ERR_CUDA;
  return NRSENSE_OK;
}

}  // extern "C"
