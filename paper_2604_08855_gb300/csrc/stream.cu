// stream.cu -- neighbour enumeration on the uniform cell grid.
//
// Paper, "Implementation": for each pivot, find all neighbours by scanning the
// spatial index over the search range.  Here one warp owns one primary and
// walks the x-rows of grid cells that intersect its ball r < r_max: each row
// is one contiguous run of cell-sorted points, read with coalesced 16-byte
// loads, 32 candidates per step.  Every candidate gets its exact radial bin:
// float32 r from the fixed-point separation, and, for the rare candidates
// within float rounding of an edge, the exact integer r^2 against exact
// thresholds.
//
// Two passes per chunk of primaries:
//   count: pairs per (primary, bin)  -> counts (then an exclusive scan on the
//          host stream gives each (primary, bin) list its start)
//   fill:  each pair's neighbour index written into its (primary, bin) list,
//          in stream order (match_any ranks lanes that share a bin)
// The kernel holds few registers, so many warps per SM hide the load latency
// that dominates this phase.
#include "ctb_internal.cuh"

namespace ctb {

__device__ __forceinline__ float slab_dist(int d, float fr) {
  return d > 0 ? (float)d - fr : (d < 0 ? (float)(-d - 1) + fr : 0.f);
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

template <bool FILL>
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
  const float R2 = g.rcell * g.rcell;
  const int K = (int)floorf(g.rcell) + 1;
  int W = 2 * K + 1, off0 = -K;
  bool fullwin = false;
  if (g.periodic && W >= (int)nc) {
    W = (int)nc;
    off0 = -(((int)nc - 1) / 2);
    fullwin = true;
  }
  const int nrows = W * W;
  const uint64_t lowmask = (1ull << g.shift) - 1ull;
  const float frac_scale = 1.0f / (float)(1ull << g.shift);
  unsigned long long my_pairs = 0;

  while (true) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(a.work, 1ull);
    i = __shfl_sync(0xffffffffu, i, 0);
    if (i >= (unsigned long long)a.prim_count) break;
    const int64_t gi = a.prim_begin + (int64_t)i;
    const uint32_t sp = a.prim ? __ldg(a.prim + gi) : (uint32_t)gi;
    const uint4 P = __ldg(a.pts + sp);
    // batch: the primary's catalogue owns cells [cat * ncells, (cat + 1) * ncells)
    const uint32_t cbase = a.keys ? (__ldg(a.keys + sp) / g.ncells) * g.ncells : 0u;
    if (!FILL && lane == 0) a.wprim[i] = __uint_as_float(P.w);
    const uint64_t ib = i * (uint64_t)nbins;
    if (FILL) {
      for (int b = lane; b < nbins; b += 32) cnt[b] = __ldg(a.offsets + ib + b);
    } else {
      for (int b = 0; b < nbins; ++b) cnt[b * 32 + lane] = 0u;
    }
    __syncwarp();

    const uint64_t sx = (uint64_t)P.x * nc, sy = (uint64_t)P.y * nc, sz = (uint64_t)P.z * nc;
    const int cxp = (int)(sx >> g.shift), cyp = (int)(sy >> g.shift), czp = (int)(sz >> g.shift);
    const float fry = (float)(sy & lowmask) * frac_scale;
    const float frz = (float)(sz & lowmask) * frac_scale;
    const float fx = (float)cxp + (float)(sx & lowmask) * frac_scale;

    for (int t0 = 0; t0 < nrows; t0 += 32) {
      // ---- this lane's row: up to two point ranges (periodic wrap in x)
      const int t = t0 + lane;
      uint32_t s0 = 0, e0 = 0, s1 = 0, e1 = 0;
      if (t < nrows) {
        const int dy = t % W + off0, dz = t / W + off0;
        float gy = slab_dist(dy, fry), gz = slab_dist(dz, frz);
        if (fullwin) {
          gy = fminf(gy, fminf(slab_dist(dy - (int)nc, fry), slab_dist(dy + (int)nc, fry)));
          gz = fminf(gz, fminf(slab_dist(dz - (int)nc, frz), slab_dist(dz + (int)nc, frz)));
        }
        const float rho2 = gy * gy + gz * gz;
        int cy = cyp + dy, cz = czp + dz;
        bool ok = rho2 < R2;
        if (g.periodic) {
          cy = pmod(cy, (int)nc);
          cz = pmod(cz, (int)nc);
        } else {
          ok = ok && cy >= 0 && cy < (int)nc && cz >= 0 && cz < (int)nc;
        }
        if (ok) {
          const float hw = sqrtf(R2 - rho2);
          int lo = (int)floorf(fx - hw), hi = (int)floorf(fx + hw);
          const uint32_t rb = cbase + ((uint32_t)cz * nc + (uint32_t)cy) * nc;
          int a0 = 1, b0 = 0, a1 = 1, b1 = 0;
          if (g.periodic) {
            if (hi - lo + 1 >= (int)nc) {
              a0 = 0;
              b0 = (int)nc - 1;
            } else {
              const int lm = pmod(lo, (int)nc), hm = pmod(hi, (int)nc);
              a0 = lm;
              if (lm <= hm) {
                b0 = hm;
              } else {
                b0 = (int)nc - 1;
                a1 = 0;
                b1 = hm;
              }
            }
          } else {
            a0 = max(lo, 0);
            b0 = min(hi, (int)nc - 1);
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
        for (uint32_t base = cs; base < ce; base += 32) {
          const uint32_t j = base + lane;
          const bool valid = j < ce;
          const uint4 q = valid ? __ldg(a.pts + j) : P;
          const int ix = (int)(q.x - P.x), iy = (int)(q.y - P.y), iz = (int)(q.z - P.z);
          const float dx = __int2float_rn(ix), dy = __int2float_rn(iy), dz = __int2float_rn(iz);
          const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
          bool inb = valid && r2 > 0.f && r2 >= g.rlo2_u && r2 < g.rhi2_u;
          int b = 0;
          if (inb) {
            const float r = r2 * rsqrtf(r2);
            const float tt = (r - g.rmin_u) * g.inv_dr_u;
            b = (int)floorf(tt);
            const float fr = tt - (float)b;
            if (b < 0 || b >= nbins || fr < 1e-4f || fr > 1.f - 1e-4f) {
              // within float rounding of an edge: exact integer r^2 vs exact thresholds
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
          if (FILL) {
            const unsigned act = __ballot_sync(0xffffffffu, inb);
            if (inb) {
              const unsigned grp = __match_any_sync(act, b);
              const unsigned rank = __popc(grp & lt);
              const uint32_t c0 = cnt[b];
              __syncwarp(act);
              a.lists[(uint64_t)c0 + rank] = j;
              if (rank == 0) cnt[b] = c0 + __popc(grp);
            }
            __syncwarp();
          } else if (inb) {
            cnt[b * 32 + lane] += 1u;  // lane-private: no ordering, no conflict
          }
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

int stream_blocks_per_sm(bool fill, int nbins) {
  int nb = 0;
  const size_t smem = stream_smem(fill, nbins);
  if (!fill && smem > 48 * 1024 &&
      cudaFuncSetAttribute(k_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  cudaError_t e = fill ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream<true>, kStreamThreads, smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_stream<false>, kStreamThreads, smem);
  return e == cudaSuccess ? nb : 0;
}

cudaError_t launch_stream(const StreamArgs& a, bool fill, int nblocks, cudaStream_t st) {
  const size_t smem = stream_smem(fill, a.g.nbins);
  if (!fill && smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_stream<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (fill)
    k_stream<true><<<nblocks, kStreamThreads, smem, st>>>(a);
  else
    k_stream<false><<<nblocks, kStreamThreads, smem, st>>>(a);
  ++g_launches;
  return cudaGetLastError();
}

}  // namespace ctb
