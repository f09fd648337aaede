// stream.cu -- neighbour enumeration on the uniform cell grid.
//
// Paper, "Implementation": for each pivot, find all neighbours by scanning the
// spatial index over the search range.  Here one warp owns one primary and
// walks the x-rows of grid cells that intersect its ball r < r_max: each row
// is one contiguous run of cell-sorted points, read with coalesced 16-byte
// loads, 32 candidates per step.  Rows are split finer along x than across
// (kXSub), so a row's range ends close to the ball; in sphere mode a row is
// also cut to the shell that holds the points.  Every candidate gets its exact radial bin:
// float32 r from the fixed-point separation, and, for the rare candidates
// within float rounding of an edge, the exact integer r^2 against exact
// thresholds.
//
// Two passes per chunk of primaries:
//   count: pairs per (primary, bin)  -> counts (then an exclusive scan on the
//          host stream gives each (primary, bin) list its start); the bin of
//          every candidate is also stored as one byte (kNoBin: not a pair):
//          each block of 32 rows takes a range of its warp's pool in the code
//          buffer, and each cell-row segment in it starts on a 4-byte boundary
//   fill:  walks the same candidate stream, reads the stored bin codes four
//          per lane (no point loads, no distances) and writes each pair's
//          neighbour index into its (primary, bin) list (match_any ranks the
//          lanes that share a bin)
// The kernel holds few registers, so many warps per SM hide the load latency
// that dominates this phase.
#include <algorithm>

#include "ctb_internal.cuh"

namespace ctb {

__device__ __forceinline__ float slab_dist(int d, float fr) {
  return d > 0 ? (float)d - fr : (d < 0 ? (float)(-d - 1) + fr : 0.f);
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

constexpr uint8_t kNoBin = 0xff;  // bin code of a candidate that is not a pair
constexpr unsigned long long kCodePool = 16384;  // code bytes a warp takes at a time

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Geometry of one primary's row window, shared by both passes.
struct RowWin {
  int W, off0, nrows;
  bool fullwin;
  float R2, fx, fry, frz;  // (r_max in cell units)^2; primary's x in x-cell units, y and z fractions
  float xs;                // x-cells per cell (ncx / nc)
  int cxp, cyp, czp;
  uint32_t cbase;
};

// The point ranges of row t of the window (up to two: periodic wrap in x,
// or the two crossings of the sphere's shell); empty ranges have s >= e.
// SHELL (sphere mode): every point lies in the shell of g.shell_r2lo ..
// g.shell_r2hi around the origin, so a row that misses it is skipped without
// a load, and a row that crosses it is cut to its crossings.
template <bool SHELL>
__device__ __forceinline__ void row_ranges(const StreamArgs& a, const Geom& g, const RowWin& rw, int t, uint32_t& s0,
                                           uint32_t& e0, uint32_t& s1, uint32_t& e1) {
  const uint32_t nc = g.nc;
  s0 = e0 = s1 = e1 = 0;
  if (t >= rw.nrows) return;
  const int dy = t % rw.W + rw.off0, dz = t / rw.W + rw.off0;
  float gy = slab_dist(dy, rw.fry), gz = slab_dist(dz, rw.frz);
  if (rw.fullwin) {
    gy = fminf(gy, fminf(slab_dist(dy - (int)nc, rw.fry), slab_dist(dy + (int)nc, rw.fry)));
    gz = fminf(gz, fminf(slab_dist(dz - (int)nc, rw.frz), slab_dist(dz + (int)nc, rw.frz)));
  }
  const float rho2 = gy * gy + gz * gz;
  int cy = rw.cyp + dy, cz = rw.czp + dz;
  bool ok = rho2 < rw.R2;
  if (g.periodic) {
    cy = pmod(cy, (int)nc);
    cz = pmod(cz, (int)nc);
  } else {
    ok = ok && cy >= 0 && cy < (int)nc && cz >= 0 && cz < (int)nc;
  }
  if (!ok) return;
  // the row's x-range in x-cells (a row is split xs times finer along x
  // than across, so its ends overshoot the ball by less)
  const float hw = sqrtf(rw.R2 - rho2) * rw.xs;
  const int nx = (int)g.ncx;
  int lo = (int)floorf(rw.fx - hw), hi = (int)floorf(rw.fx + hw);
  const uint32_t rb = rw.cbase + ((uint32_t)cz * nc + (uint32_t)cy) * (uint32_t)nx;
  int a0 = 1, b0 = 0, a1 = 1, b1 = 0;
  if constexpr (SHELL) {
    // distance range from the shell's axis to the row's (y, z) cross-section
    const float ly = (float)cy - g.shell_c[1], lz = (float)cz - g.shell_c[2];
    const float ny = ly > 0.f ? ly : (ly + 1.f < 0.f ? -(ly + 1.f) : 0.f);
    const float nz = lz > 0.f ? lz : (lz + 1.f < 0.f ? -(lz + 1.f) : 0.f);
    const float fy = fmaxf(fabsf(ly), fabsf(ly + 1.f)), fz = fmaxf(fabsf(lz), fabsf(lz + 1.f));
    const float d2min = ny * ny + nz * nz, d2max = fy * fy + fz * fz;
    if (d2min >= g.shell_r2hi) return;
    // x offsets (x-cells) of the shell along the row: [alo, ahi] either side of the centre
    const float ahi = sqrtf(g.shell_r2hi - d2min) * rw.xs;
    const float alo = g.shell_r2lo > d2max ? sqrtf(g.shell_r2lo - d2max) * rw.xs : 0.f;
    const float xl = rw.fx - hw, xh = rw.fx + hw, cx = g.shell_c[0];
    // the ball's x-range meets the upper crossing [cx + alo, cx + ahi] and the lower one
    const float pl = fmaxf(xl, cx + alo), ph = fminf(xh, cx + ahi);
    const float ml = fmaxf(xl, cx - ahi), mh = fminf(xh, cx - alo);
    int ma = nx, mb = -1, pa = nx, pb = -1;
    if (ml <= mh) {
      ma = max((int)floorf(ml), 0);
      mb = min((int)floorf(mh), nx - 1);
    }
    if (pl <= ph) {
      pa = max((int)floorf(pl), 0);
      pb = min((int)floorf(ph), nx - 1);
    }
    if (ma <= mb && pa <= pb && pa <= mb + 1) {  // touching or overlapping: one range
      a0 = ma;
      b0 = max(mb, pb);
    } else if (ma <= mb) {
      a0 = ma;
      b0 = mb;
      a1 = pa;
      b1 = pb;
    } else {
      a0 = pa;
      b0 = pb;
    }
  } else if (g.periodic) {
    if (hi - lo + 1 >= nx) {
      a0 = 0;
      b0 = nx - 1;
    } else {
      const int lm = pmod(lo, nx), hm = pmod(hi, nx);
      a0 = lm;
      if (lm <= hm) {
        b0 = hm;
      } else {
        b0 = nx - 1;
        a1 = 0;
        b1 = hm;
      }
    }
  } else {
    a0 = max(lo, 0);
    b0 = min(hi, nx - 1);
  }
  if (a0 <= b0) {
    s0 = __ldg(a.cell_start + rb + a0);
    e0 = __ldg(a.cell_start + rb + b0 + 1);
  }
  if (a1 <= b1) {
    s1 = __ldg(a.cell_start + rb + a1);
    e1 = __ldg(a.cell_start + rb + b1 + 1);
  }
}

// GEN: sphere mode -- bin edges not linear in r (the angle bins, count
// pass) and rows cut to the points' shell (both passes)
template <bool FILL, bool GEN>
__global__ void __launch_bounds__(kStreamThreads) k_stream(StreamArgs a) {
  extern __shared__ uint32_t s_cnt_all[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const Geom g = a.g;
  const int nbins = g.nbins;
  // fill: running list position per bin; count: lane-private histogram hist[b * 32 + lane]
  uint32_t* cnt = s_cnt_all + warp * (FILL ? kNbinsCap : nbins * 32);
  const unsigned lt = (1u << lane) - 1u;
  const uint32_t nc = g.nc;
  RowWin rw;
  rw.R2 = g.rcell * g.rcell;
  rw.xs = (float)(g.ncx / nc);
  {
    const RowWindow win = row_window(g);
    rw.W = win.W;
    rw.off0 = win.off0;
    rw.fullwin = win.fullwin;
  }
  rw.nrows = rw.W * rw.W;
  const int nrb = (rw.nrows + 31) / 32;
  const uint64_t lowmask = (1ull << g.shift) - 1ull;
  const float frac_scale = 1.0f / (float)(1ull << g.shift);
  unsigned long long my_pairs = 0;
  // count: this warp's pool in the code buffer (row blocks take consecutive
  // ranges of it; a new pool is taken when one does not fit)
  unsigned long long pool = 0, pool_end = 0;

  while (true) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(a.work, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= (unsigned long long)a.prim_count) break;
    const int64_t gi = a.prim_begin + (int64_t)i;
    const uint32_t sp = a.prim ? __ldg(a.prim + gi) : (uint32_t)gi;
    const uint4 P = __ldg(a.pts + sp);
    // batch: the primary's catalogue owns cells [cat * ncells, (cat + 1) * ncells)
    rw.cbase = a.keys ? (__ldg(a.keys + sp) / g.ncells) * g.ncells : 0u;
    if (!FILL && lane == 0) a.wprim[i] = a.wsub ? __ldg(a.wsub + gi) : __uint_as_float(P.w);
    const uint64_t ib = i * (uint64_t)nbins;
    if (FILL) {
      for (int b = lane; b < nbins; b += 32) cnt[b] = __ldg(a.offsets + ib + b);
    } else {
      for (int b = 0; b < nbins; ++b) cnt[b * 32 + lane] = 0u;
    }
    __syncwarp();

    const uint64_t sx = (uint64_t)P.x * g.ncx, sy = (uint64_t)P.y * nc, sz = (uint64_t)P.z * nc;
    rw.cxp = (int)(sx >> g.shift);
    rw.cyp = (int)(sy >> g.shift);
    rw.czp = (int)(sz >> g.shift);
    rw.fry = (float)(sy & lowmask) * frac_scale;
    rw.frz = (float)(sz & lowmask) * frac_scale;
    rw.fx = (float)rw.cxp + (float)(sx & lowmask) * frac_scale;

    for (int t0 = 0, rb = 0; t0 < rw.nrows; t0 += 32, ++rb) {
      uint32_t s0, e0, s1, e1;
      row_ranges<GEN>(a, g, rw, t0 + lane, s0, e0, s1, e1);
      // this row block's range of the code buffer: its segments in the order
      // below, each padded to a multiple of 4 codes
      unsigned long long span = (s0 < e0 ? (e0 - s0 + 3u) & ~3u : 0u) + (s1 < e1 ? (e1 - s1 + 3u) & ~3u : 0u);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) span += __shfl_xor_sync(0xffffffffu, span, o);
      unsigned long long pos = 0;
      bool codes_ok = true;
      if (FILL) {
        pos = __ldg(a.code_base + i * (uint64_t)nrb + rb);
        // the block's codes to L2 ahead of the segment loads (one line per lane)
        for (unsigned long long ln = (unsigned long long)lane * 128u; ln < span; ln += 32u * 128u)
          prefetch_l2(a.codes + pos + ln);
      } else {
        if (pool + span > pool_end) {
          const unsigned long long take = span > kCodePool ? span : kCodePool;
          if (lane == 0) pool = atomicAdd(a.code_total, take);
          pool = __shfl_sync(0xffffffffu, pool, 0);
          pool_end = pool + take;
        }
        pos = pool;
        pool += span;
        if (lane == 0) a.code_base[i * (uint64_t)nrb + rb] = pos;
        // past the buffer: counts stay exact, codes are dropped and the host
        // grows the buffer and counts the chunk again
        codes_ok = pos + span <= a.code_cap;
      }
      if constexpr (FILL) {
        // The row block's codes are one contiguous run: lane t's segments
        // in order, each padded to 4 codes.  Walk it as a stream, lane l
        // taking code word k0 + l (4 candidates of one segment), with the
        // next step's word loaded ahead.
        const uint32_t len0 = s0 < e0 ? (e0 - s0 + 3u) & ~3u : 0u;
        const uint32_t len1 = s1 < e1 ? (e1 - s1 + 3u) & ~3u : 0u;
        uint32_t incl = len0 + len1;  // inclusive prefix of the padded lengths over the lanes
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const uint32_t excl = incl - len0 - len1;
        const uint32_t nwords = (uint32_t)(span >> 2);
        const uint32_t* rbw = reinterpret_cast<const uint32_t*>(a.codes + pos);
        uint32_t word = (uint32_t)lane < nwords ? __ldcs(rbw + lane) : 0xffffffffu;
        for (uint32_t k0 = 0; k0 < nwords; k0 += 32) {
          const uint32_t kn = k0 + 32u + (uint32_t)lane;
          const uint32_t wnext = kn < nwords ? __ldcs(rbw + kn) : 0xffffffffu;
          // the segment of code 4 (k0 + lane): first lane t with incl_t above it
          const uint32_t cpos = 4u * (k0 + (uint32_t)lane);
          int t = 0;
#pragma unroll
          for (int st = 16; st > 0; st >>= 1)
            if (__shfl_sync(0xffffffffu, incl, t + st - 1) <= cpos) t += st;
          const uint32_t r = cpos - __shfl_sync(0xffffffffu, excl, t);
          const uint32_t l0 = __shfl_sync(0xffffffffu, len0, t);
          const uint32_t sa0 = __shfl_sync(0xffffffffu, s0, t), ea0 = __shfl_sync(0xffffffffu, e0, t);
          const uint32_t sa1 = __shfl_sync(0xffffffffu, s1, t), ea1 = __shfl_sync(0xffffffffu, e1, t);
          const bool first = r < l0;
          const uint32_t jb = first ? sa0 + r : sa1 + (r - l0);
          const uint32_t je = first ? ea0 : ea1;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const uint32_t j = jb + (uint32_t)k;
            const uint32_t code = (word >> (8 * k)) & 0xffu;
            // words past the run read as all kNoBin; the padding after a
            // segment's end holds no codes
            const bool inb = code != kNoBin && j < je;
            const int b = (int)code;
            const unsigned act = __ballot_sync(0xffffffffu, inb);
            if (inb) {
              const unsigned grp = __match_any_sync(act, b);
              const unsigned rank = __popc(grp & lt);
              const uint32_t c0 = cnt[b];
              __syncwarp(act);
              __stcs(a.lists + ((uint64_t)c0 + rank), j);
              if (rank == 0) cnt[b] = c0 + __popc(grp);
            }
            __syncwarp();
          }
          word = wnext;
        }
        continue;
      }
      unsigned pend = __ballot_sync(0xffffffffu, s0 < e0 || s1 < e1);
      while (pend) {
        // ---- next segment (warp-uniform)
        const int src = __ffs(pend) - 1;
        const bool h0 = __shfl_sync(0xffffffffu, s0 < e0, src);
        const uint32_t cs = __shfl_sync(0xffffffffu, h0 ? s0 : s1, src);
        const uint32_t ce = __shfl_sync(0xffffffffu, h0 ? e0 : e1, src);
        if (lane == src) {
          if (h0) s0 = e0;
          else s1 = e1;
        }
        pend = __ballot_sync(0xffffffffu, s0 < e0 || s1 < e1);
        const unsigned long long seg0 = pos;  // code of candidate j: codes[seg0 + (j - cs)]
        pos += (ce - cs + 3u) & ~3u;
        for (uint32_t base = cs; base < ce; base += 32) {
          const uint32_t j = base + lane;
          const bool valid = j < ce;
          // lanes past the segment load its last point and are masked by `valid`
          const uint4 q = __ldg(a.pts + (valid ? j : ce - 1u));
          const int ix = (int)(q.x - P.x), iy = (int)(q.y - P.y), iz = (int)(q.z - P.z);
          const float dx = __int2float_rn(ix), dy = __int2float_rn(iy), dz = __int2float_rn(iz);
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          // rlo2_u > 0 also excludes r = 0 (coincident points)
          bool inb = valid && r2 >= g.rlo2_u && r2 < g.rhi2_u;
          int b = 0;
          if (inb) {
            const float r = r2 * rsqrtf(r2);
            float tt, guard;
            if constexpr (GEN) {
              // sphere: the bin of theta = 2 asin(chord / 2).  Its float
              // error stays below 1e-6 theta while chord / 2 <= 0.99 (asin
              // is ill-conditioned towards 1); the guard is ten times that,
              // and larger chords always take the exact test.  Up to
              // chord / 2 = 1/8 (theta 14 degrees) the Maclaurin series of
              // asin to x^7 serves: truncation below 2e-9 theta, float
              // evaluation below 2e-7 theta.
              const float x = r * g.half_unit;
              float th;
              if (x <= 0.125f) {
                const float x2 = x * x;
                th = 2.f * x * fmaf(x2, fmaf(x2, fmaf(x2, 5.f / 112.f, 3.f / 40.f), 1.f / 6.f), 1.f);
              } else {
                th = 2.f * asinf(fminf(x, 1.f));
              }
              tt = (th - g.tmin) * g.inv_dt;
              guard = x > 0.99f ? 1.f : fmaxf(1e-4f, fmaf(1e-5f, th, 1e-7f) * g.inv_dt);
            } else {
              tt = (r - g.rmin_u) * g.inv_dr_u;
              guard = 1e-4f;
            }
            b = (int)floorf(tt);
            const float fr = tt - (float)b;
            if ((unsigned)b >= (unsigned)nbins || fabsf(fr - 0.5f) > 0.5f - guard) {
              // within float rounding of an edge: exact integer r^2 vs
              // exact thresholds
              const unsigned long long e2 = (unsigned long long)((long long)ix * ix + (long long)iy * iy +
                                                                 (long long)iz * iz);
              if (e2 == 0ull || e2 < __ldg(a.thr) || e2 >= __ldg(a.thr + nbins)) {
                inb = false;
              } else {
                b = min(max(b, 0), nbins - 1);
                while (e2 < __ldg(a.thr + b)) --b;
                while (e2 >= __ldg(a.thr + b + 1)) ++b;
              }
            }
          }
          if (valid && codes_ok) __stcs(a.codes + (seg0 + (j - cs)), inb ? (unsigned char)b : (unsigned char)kNoBin);
          if (inb) cnt[b * 32 + lane] += 1u;  // lane-private: no ordering, no conflict
        }
      }
    }
    if (!FILL) {
      __syncwarp();
      for (int b = lane; b < nbins; b += 32) {
        uint32_t s = 0;
        for (int k = 0; k < 32; ++k) s += cnt[b * 32 + ((b + k) & 31)];  // rotated: no bank conflict
        a.counts[ib + b] = s;
        my_pairs += s;
      }
    }
    __syncwarp();
  }
  if (!FILL) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, o);
    if (lane == 0 && my_pairs) atomicAdd(a.total, my_pairs);
  }
}

static size_t stream_smem(bool fill, int nbins) {
  return (size_t)(kStreamThreads / 32) * (fill ? kNbinsCap : nbins * 32) * sizeof(uint32_t);
}

int stream_blocks_per_sm(bool fill, int nbins, bool general) {
  const void* fn = fill ? (general ? (const void*)k_stream<true, true> : (const void*)k_stream<true, false>)
                        : (general ? (const void*)k_stream<false, true> : (const void*)k_stream<false, false>);
  const size_t smem = stream_smem(fill, nbins);
  if (smem > 48 * 1024 && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int nb = 0;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kStreamThreads, smem) == cudaSuccess ? nb : 0;
}

cudaError_t launch_stream(const StreamArgs& a, bool fill, int nblocks, cudaStream_t st) {
  const size_t smem = stream_smem(fill, a.g.nbins);
  const bool gen = a.g.general != 0;
  const void* fn = fill ? (gen ? (const void*)k_stream<true, true> : (const void*)k_stream<true, false>)
                        : (gen ? (const void*)k_stream<false, true> : (const void*)k_stream<false, false>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (fill && gen)
    k_stream<true, true><<<nblocks, kStreamThreads, smem, st>>>(a);
  else if (fill)
    k_stream<true, false><<<nblocks, kStreamThreads, smem, st>>>(a);
  else if (gen)
    k_stream<false, true><<<nblocks, kStreamThreads, smem, st>>>(a);
  else
    k_stream<false, false><<<nblocks, kStreamThreads, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
