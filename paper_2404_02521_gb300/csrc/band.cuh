// Cluster band layout shared by the fine and coarse kernels.
//
// A state of M x M nodes is split over a cluster of C CTAs: CTA `rank` owns band rows
// j = rank*BH .. rank*BH + BH - 1 (BH = G*K) and NCOL >= M columns.  Every shared-memory
// plane of a band holds BH + 2 rows: plane row 0 is a copy of the last row of CTA rank-1,
// plane rows 1..BH are the CTA's own rows, plane row BH + 1 is a copy of the first row of
// CTA rank+1.  A CTA that writes its first or last own row also stores the value into the
// neighbour's halo row (a distributed-shared-memory store, issued before the cluster
// barrier that publishes it), so every stencil read is a local shared-memory load.
// Halo rows outside the domain stay zero; the coefficients that would read them vanish
// (y = 0) or the row is not a PDE row (y = ymax).
//
// Thread t owns column t % NCOL and the K band rows (t / NCOL)*K .. +K-1.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace bsp {

namespace cg = cooperative_groups;

template <int NCOL_, int NT_, int K_>
struct BandCfg {
  static constexpr int NCOL = NCOL_;
  static constexpr int NT = NT_;
  static constexpr int K = K_;
  static constexpr int G = NT / NCOL;
  static constexpr int BH = G * K;
  static constexpr int PLANE = (BH + 2) * NCOL;   // floats per plane including halo rows
  static constexpr int NW = NT / 32;
};

// Remote halo targets of one plane: the neighbours' halo rows that mirror this CTA's
// first and last own rows (nullptr at the ends of the cluster).
struct HaloPush {
  float* prev_bottom;   // rank-1's plane row BH+1
  float* next_top;      // rank+1's plane row 0
};

template <class CFG>
__device__ __forceinline__ HaloPush halo_push(cg::cluster_group& cl, float* plane, int rank, int C) {
  HaloPush h;
  h.prev_bottom = rank > 0 ? cl.map_shared_rank(plane, rank - 1) + (CFG::BH + 1) * CFG::NCOL : nullptr;
  h.next_top = rank < C - 1 ? cl.map_shared_rank(plane, rank + 1) : nullptr;
  return h;
}

// Store v at own band row r (0-based), column c of a plane, mirroring rows 0 and BH-1.
template <class CFG>
__device__ __forceinline__ void band_store(float* plane, const HaloPush& h, int r, int c, float v) {
  plane[(r + 1) * CFG::NCOL + c] = v;
  if (r == 0 && h.prev_bottom) h.prev_bottom[c] = v;
  if (r == CFG::BH - 1 && h.next_top) h.next_top[c] = v;
}

// Load a state into a plane: own rows and both halo rows straight from global memory.
template <class CFG>
__device__ __forceinline__ void band_load(float* plane, const float* src, int M, int jbase, int tid) {
  for (int e = tid; e < CFG::PLANE; e += CFG::NT) {
    const int pr = e / CFG::NCOL, c = e % CFG::NCOL;
    const int j = jbase + pr - 1;
    plane[e] = (j >= 0 && j < M && c < M) ? src[(size_t)j * M + c] : 0.f;
  }
}

// Far-field values at tau for this band's Dirichlet nodes (column M-1 of every own row and,
// in the band that holds it, row M-1), one evaluation per thread, mirrored into the
// neighbours' halo rows.
template <class CFG>
__device__ __forceinline__ void band_far_field(float* plane, const HaloPush& hp, const PayoffF& pf,
                                               float tau, float h, int M, int jbase, int tid) {
  const bool has_last_row = (jbase <= M - 1) && (M - 1 < jbase + CFG::BH);
  const int n_entries = CFG::BH + (has_last_row ? (M - 1) : 0);
  for (int e = tid; e < n_entries; e += CFG::NT) {
    int r, c;
    if (e < CFG::BH) {
      r = e;
      c = M - 1;
      if (jbase + r > M - 1) continue;
    } else {
      r = M - 1 - jbase;
      c = e - CFG::BH;
    }
    band_store<CFG>(plane, hp, r, c, far_field(pf, c * h, (jbase + r) * h, tau));
  }
}

__device__ __forceinline__ void cluster_barrier(cg::cluster_group& cl, int C) {
  if (C > 1) cl.sync(); else __syncthreads();
}

}  // namespace bsp
