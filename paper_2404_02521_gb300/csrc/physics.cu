// PDE term of the PINO training loss (Sec. 3.5, eq. bs_totalloss) on the device.
//
// A coarse-propagator prediction u~ of u(tau + dtau) from u(tau) is scored by the residual of
// eq. (bse_change_variable), discretised by eq. (fd) with the slice as one implicit step, at
// the collocation points that carry a PDE row (0 <= i, j <= M-2):
//   r = (u~ - u_prev) / dtau - R_h u~ = ((u~ - u_prev) - dtau R_h u~) / dtau,
//   loss = (1/n) sum r^2  (n = (M-1)^2),   d loss / d u~_i = (2/n) sum_j r_j d r_j / d u~_i.
// Row j of R_h reads the 3 x 3 nodes around j, so the gradient at node i gathers the residuals
// of the (up to) nine collocation points around i, each recomputed from u~; no scratch plane
// is needed.  The residual is evaluated in FP32 from the same index-unit coefficients as the
// steppers (dtau R_h with the slice's dtau), the loss accumulated in FP64.
#include "common.cuh"

namespace bsp {

namespace {

struct PhysItem {
  const float* pred;
  const float* prev;
  float* grad;     // nullptr: loss only
  double* loss;    // device
  ItemDesc d;      // coefficients of dtau R_h
  float rdtau;     // 1 / dtau
};

constexpr int kPhysMaxItems = 32;
constexpr int kPhysThreads = 256;

struct PhysBatch {
  PhysItem it[kPhysMaxItems];
  int M;
  double inv_n;
};

// Coefficients of row (i, j) of dtau R_h: east, west, south (j + 1), north (j - 1), cross.
struct RowW {
  float e, w, s, n, g, rdt;
};

__device__ __forceinline__ RowW row_weights(const ItemDesc& d, int i, int j) {
  RowW c;
  float cgi, gj;
  column_coefs(d, i, c.e, c.w, cgi);
  row_coefs(d, j, c.s, c.n, gj);
  c.g = cgi * gj;
  c.rdt = d.rdt;
  return c;
}

// r at collocation point (i, j).  Neighbours at x = 0 or y = 0 are read clamped: their
// weights vanish there.
__device__ __forceinline__ float residual_at(const PhysItem& it, int M, int i, int j) {
  const float* u = it.pred;
  const int il = i > 0 ? i - 1 : 0, ir = i + 1, jn = j > 0 ? j - 1 : 0, js = j + 1;
  const RowW c = row_weights(it.d, i, j);
  const float nW = u[jn * M + il], nC = u[jn * M + i], nE = u[jn * M + ir];
  const float cW = u[j * M + il], cC = u[j * M + i], cE = u[j * M + ir];
  const float sW = u[js * M + il], sC = u[js * M + i], sE = u[js * M + ir];
  // dtau R_h u~ (eq. fd in index units)
  const float t = c.e * (cE - cC) - c.w * (cC - cW) + c.s * (sC - cC) - c.n * (cC - nC) +
                  c.g * ((sE - nE) - (sW - nW)) - c.rdt * cC;
  return ((cC - it.prev[j * M + i]) - t) * it.rdtau;
}

// Weight with which row (i, j) of dtau R_h reads its neighbour at offset (di, dj).
__device__ __forceinline__ float weight_at(const RowW& c, int di, int dj) {
  if (di == 0 && dj == 0) return -(c.e + c.w + c.s + c.n + c.rdt);
  if (dj == 0) return di > 0 ? c.e : c.w;
  if (di == 0) return dj > 0 ? c.s : c.n;
  return di == dj ? c.g : -c.g;   // (+1,+1), (-1,-1): +g; (+1,-1), (-1,+1): -g
}

__global__ void __launch_bounds__(kPhysThreads) physics_loss_kernel(const __grid_constant__ PhysBatch pb) {
  const PhysItem& it = pb.it[blockIdx.y];
  const int M = pb.M;
  const int node = blockIdx.x * kPhysThreads + threadIdx.x;
  double r2 = 0.0;
  if (node < M * M) {
    const int i = node % M, j = node / M;
    const bool colloc = i <= M - 2 && j <= M - 2;
    float own = 0.f;
    if (colloc) {
      own = residual_at(it, M, i, j);
      r2 = (double)own * (double)own;
    }
    if (it.grad) {
      // d r_q / d u~_node = (delta - w_q(node - q)) / dtau over the collocation points q
      // around the node
      float acc = 0.f;
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const int qi = i - di, qj = j - dj;   // the node is q's neighbour at (di, dj)
          if (qi < 0 || qj < 0 || qi > M - 2 || qj > M - 2) continue;
          const float rq = (di == 0 && dj == 0) ? own : residual_at(it, M, qi, qj);
          const float w = weight_at(row_weights(it.d, qi, qj), di, dj);
          acc = fmaf(rq, ((di == 0 && dj == 0) ? 1.f : 0.f) - w, acc);
        }
      }
      it.grad[node] = (float)(2.0 * pb.inv_n) * acc * it.rdtau;
    }
  }
  // block sum of r^2 (FP64), one atomic per block
  __shared__ double part[kPhysThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) r2 += __shfl_down_sync(0xffffffffu, r2, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = r2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kPhysThreads / 32; ++w) s += part[w];
    if (s != 0.0) atomicAdd(it.loss, s * pb.inv_n);
  }
}

}  // namespace

int launch_physics_loss(const bs_grid* g, const bs_params* p, const float* const* u_pred,
                        const float* const* u_prev, const double* dtau, int B, double* loss,
                        float* const* grad, cudaStream_t s) {
  const int M = g->M;
  PhysBatch pb;
  pb.M = M;
  pb.inv_n = 1.0 / ((double)(M - 1) * (double)(M - 1));
  BS_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(double) * (size_t)B, s));
  const unsigned blocks = (unsigned)(((size_t)M * M + kPhysThreads - 1) / kPhysThreads);
  for (int base = 0; base < B; base += kPhysMaxItems) {
    const int nb = B - base < kPhysMaxItems ? B - base : kPhysMaxItems;
    for (int k = 0; k < nb; ++k) {
      const int b = base + k;
      PhysItem& it = pb.it[k];
      it.pred = u_pred[b];
      it.prev = u_prev[b];
      it.grad = grad ? grad[b] : nullptr;
      it.loss = loss + b;
      it.d = make_item(p[b], 0.0, dtau[b]);
      it.rdtau = (float)(1.0 / dtau[b]);
    }
    physics_loss_kernel<<<dim3(blocks, (unsigned)nb), kPhysThreads, 0, s>>>(pb);
    BS_CUDA_TRY(cudaGetLastError());
  }
  return BS_OK;
}

}  // namespace bsp
