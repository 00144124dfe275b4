// K3 + K4: the PINO coarse propagator (Sec. 3.4-3.5) on tensor cores, and bilinear
// resampling between the state grid and the network grid.
//
// Network (reading of Sec. 3.5): input channels per node [u, x, y, tau_n, dtau, sigma1,
// sigma2, rho, r]; lifting 9 -> C; L Fourier layers v <- ReLU(K v + W v + b) where K keeps
// ky in [0, my) U [Mp-my, Mp) and kx in [0, mx) of the half spectrum and mixes channels per
// mode with a complex C x C matrix; projection C -> H -> 1 with ReLU; the output is added to
// u and the far-field data are set.  Batch normalisation is folded into W, b at load time.
//
// Every contraction runs on tcgen05 (umma.cuh), BF16 operands, FP32 accumulation:
//   G1 x-DFT      [(c,y)]  x [x]          -> (kx, re/im)         N = 32 (24 used),  K = Mp
//   G2 y-DFT      [(c,kx)] x [(y,re/im)]  -> (ky mode, re/im)    N = 64 (48 used),  K = 2 Mp
//   G3 mixing     per mode: [state] x [(c,re/im)] -> (o,re/im)   N = 64, K = 64 (complex as
//                 the real 2x2 block form of the C x C mode matrix)
//   G4 inv. y-DFT [(o,kx)] x [(ky,re/im)] -> (y, re/im)          N = 2 Mp (chunks of 64), K = 48
//   G5 inv. x-DFT [pixel: x] x [(kx,re/im) of (o,y)] -> o, Hermitian weights and 1/Mp^2,
//      + pointwise [pixel] x [c] -> o, both into one accumulator (K = 32 each); the
//                 epilogue adds the bias and applies ReLU
//      At Mp = 128 a tile is one row of pixels; before the last layer the same kernel then
//      runs the next layer's G1 on the row (pino_pointwise_xdft_kernel), so only the first
//      layer launches G1 on its own.
//   P  projection [pixel]  x [c]          -> hidden, epilogue ReLU . w2 + b2, residual
// Each epilogue writes the K-contiguous layout the next GEMM reads, so no transposes run
// between them.  The DFT matrices are exact transforms (not learned) stored in BF16.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "umma.cuh"

namespace bsp {

struct PinoState {
  const float* in;     // state on its own grid (M x M)
  float* out;          // PROP: output on the same grid
  int M;
  float h;             // grid spacing of in/out
  float tau, dtau;     // network time inputs
  float s1, s2, rho, r;
  PayoffF pf;
};

enum { PAPPLY_PROP = 0, PAPPLY_INIT = 1, PAPPLY_ITER = 2, PAPPLY_ITER_SKIP = 3 };

struct PinoRes {
  int Mp = 0, cap = 0, st_cap = 0;
  bf16 *Ex = nullptr, *Ey = nullptr, *Eyi = nullptr, *Exi = nullptr;
  bf16 *act_cp = nullptr, *act_pc = nullptr, *X1 = nullptr, *X2 = nullptr, *Y = nullptr, *Z1 = nullptr;
  float *wout = nullptr, *ump = nullptr;
  PinoState* st = nullptr;
};

}  // namespace bsp

struct bs_pino {
  int cin, C, mx, my, L, H;
  float* lift_w;   // [cin][C]
  float* lift_b;   // [C]
  bsp::bf16* R;    // [L][MY*mx][64][64]
  bsp::bf16* Wpw;  // [L][C][C]  (o, c)
  float* pw_b;     // [L][C]
  bsp::bf16* W1;   // [H][C]
  float* b1;       // [H]
  float* w2;       // [H]
  float b2;
  int* err;
  bsp::PinoRes res[2];
};

namespace bsp {

static int dev_alloc(void** p, size_t bytes) {
  note_device_alloc();
  BS_CUDA_TRY(cudaMalloc(p, bytes));
  return BS_OK;
}

template <class T>
static int upload(T** d, const std::vector<T>& h) {
  int rc = dev_alloc((void**)d, h.size() * sizeof(T));
  if (rc) return rc;
  BS_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return BS_OK;
}

static bf16 to_bf16(double x) { return __float2bfloat16((float)x); }

// ---------------------------------------------------------------------------------------
// Exact DFT matrices for a network grid Mp (host, FP64 -> BF16)
// ---------------------------------------------------------------------------------------
static int build_dft(bs_pino* net, PinoRes& R) {
  const int Mp = R.Mp, mx = net->mx, my = net->my, MY = 2 * my;
  const double tp = 2.0 * M_PI;
  auto ky_of = [&](int q) { return q < my ? q : Mp - MY + q; };
  std::vector<bf16> Ex((size_t)32 * Mp, to_bf16(0)), Ey((size_t)64 * 2 * Mp, to_bf16(0)),
      Eyi((size_t)2 * Mp * 48, to_bf16(0)), Exi((size_t)Mp * 32, to_bf16(0));
  for (int kx = 0; kx < mx; ++kx)
    for (int x = 0; x < Mp; ++x) {
      const double ph = tp * ((double)kx * x / Mp);
      Ex[(size_t)(2 * kx) * Mp + x] = to_bf16(std::cos(ph));
      Ex[(size_t)(2 * kx + 1) * Mp + x] = to_bf16(-std::sin(ph));
      const double w = (kx == 0 ? 1.0 : 2.0) / ((double)Mp * Mp);
      Exi[(size_t)x * 32 + 2 * kx] = to_bf16(w * std::cos(ph));
      Exi[(size_t)x * 32 + 2 * kx + 1] = to_bf16(-w * std::sin(ph));
    }
  for (int q = 0; q < MY; ++q)
    for (int y = 0; y < Mp; ++y) {
      const double th = tp * ((double)((long long)ky_of(q) * y % Mp) / Mp);
      const double c = std::cos(th), s = std::sin(th);
      // forward (e^{-i th}): re = a c + b s, im = b c - a s
      Ey[(size_t)(2 * q) * 2 * Mp + 2 * y] = to_bf16(c);
      Ey[(size_t)(2 * q) * 2 * Mp + 2 * y + 1] = to_bf16(s);
      Ey[(size_t)(2 * q + 1) * 2 * Mp + 2 * y] = to_bf16(-s);
      Ey[(size_t)(2 * q + 1) * 2 * Mp + 2 * y + 1] = to_bf16(c);
      // inverse (e^{+i th}): re = a c - b s, im = a s + b c
      Eyi[(size_t)(2 * y) * 48 + 2 * q] = to_bf16(c);
      Eyi[(size_t)(2 * y) * 48 + 2 * q + 1] = to_bf16(-s);
      Eyi[(size_t)(2 * y + 1) * 48 + 2 * q] = to_bf16(s);
      Eyi[(size_t)(2 * y + 1) * 48 + 2 * q + 1] = to_bf16(c);
    }
  int rc;
  if ((rc = upload(&R.Ex, Ex)) || (rc = upload(&R.Ey, Ey)) || (rc = upload(&R.Eyi, Eyi)) ||
      (rc = upload(&R.Exi, Exi)))
    return rc;
  return BS_OK;
}

static void free_res(PinoRes& R) {
  void* ptrs[] = {R.Ex, R.Ey, R.Eyi, R.Exi, R.act_cp, R.act_pc, R.X1, R.X2, R.Y, R.Z1,
                  R.wout, R.ump, R.st};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  R = PinoRes();
}

// Network-grid resources for Mp, a batch of up to B states and nst state descriptors.
static int ensure_res(bs_pino* net, int Mp, int B, int nst, PinoRes** out) {
  PinoRes& R = net->res[Mp == 128 ? 0 : 1];
  if (R.Mp == Mp && R.cap >= B && R.st_cap < nst) {
    if (R.st) cudaFree(R.st);
    R.st = nullptr;
    R.st_cap = 0;
    int rc = dev_alloc((void**)&R.st, (size_t)nst * sizeof(PinoState));
    if (rc) return rc;
    R.st_cap = nst;
  }
  if (R.Mp == Mp && R.cap >= B) {
    *out = &R;
    return BS_OK;
  }
  if (R.Mp == Mp) {   // grow the batch buffers, keep the DFT matrices
    void* keep[] = {R.Ex, R.Ey, R.Eyi, R.Exi};
    R.Ex = R.Ey = R.Eyi = R.Exi = nullptr;
    free_res(R);
    R.Ex = (bf16*)keep[0]; R.Ey = (bf16*)keep[1]; R.Eyi = (bf16*)keep[2]; R.Exi = (bf16*)keep[3];
  } else {
    free_res(R);
  }
  R.Mp = Mp;
  int rc;
  if (!R.Ex && (rc = build_dft(net, R))) return rc;
  const size_t P = (size_t)Mp * Mp, C = net->C, mx = net->mx, MY = 2 * net->my;
  const size_t Bn = (size_t)B;
  if ((rc = dev_alloc((void**)&R.act_cp, Bn * C * P * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.act_pc, Bn * C * P * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.X1, Bn * C * mx * 2 * Mp * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.X2, MY * mx * Bn * C * 2 * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.Y, Bn * C * mx * MY * 2 * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.Z1, Bn * C * Mp * mx * 2 * sizeof(bf16))) ||
      (rc = dev_alloc((void**)&R.wout, Bn * P * sizeof(float))) ||
      (rc = dev_alloc((void**)&R.ump, Bn * P * sizeof(float))) ||
      (rc = dev_alloc((void**)&R.st, (size_t)(nst > B ? nst : B) * sizeof(PinoState))))
    return rc;
  R.cap = B;
  R.st_cap = nst > B ? nst : B;
  *out = &R;
  return BS_OK;
}

// ---------------------------------------------------------------------------------------
// Epilogues (rows owned by a thread; 16 accumulator columns per chunk)
// ---------------------------------------------------------------------------------------
struct NoAcc {};

struct EpiX1 {   // G1: rows (c, y), cols (kx, re/im) -> X1[b][c][kx][y][re/im]
  typedef NoAcc Acc;
  bf16* X1; int Mp, mx, C;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc&, int, int, int) const {}
  __device__ void end(Acc&, int, int, int) const {}
  __device__ void chunk(Acc&, int b, int, int row, int c0, const float* v) const {
    if (row >= C * Mp) return;
    const int c = row / Mp, y = row - (row / Mp) * Mp;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = c0 + q;
      if (col < 2 * mx)
        X1[(((size_t)b * C + c) * mx + (col >> 1)) * (2 * Mp) + 2 * y + (col & 1)] = __float2bfloat16(v[q]);
    }
  }
};

struct EpiX2 {   // G2: rows (c, kx), cols (q, re/im) -> X2[q*mx + kx][b][c][re/im]
  typedef NoAcc Acc;
  bf16* X2; int mx, MY, C, B;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc&, int, int, int) const {}
  __device__ void end(Acc&, int, int, int) const {}
  __device__ void chunk(Acc&, int b, int, int row, int c0, const float* v) const {
    if (row >= C * mx) return;
    const int c = row / mx, kx = row - (row / mx) * mx;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = c0 + q;
      if (col < 2 * MY) {
        const int mode = (col >> 1) * mx + kx;
        X2[(((size_t)mode * B + b) * C + c) * 2 + (col & 1)] = __float2bfloat16(v[q]);
      }
    }
  }
};

struct EpiY {    // G3 (blockIdx.y = mode): rows b, cols (o, re/im) -> Y[b][o][kx][q][re/im]
  typedef NoAcc Acc;
  bf16* Y; int mx, MY, C, B;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc&, int, int, int) const {}
  __device__ void end(Acc&, int, int, int) const {}
  __device__ void chunk(Acc&, int mode, int, int row, int c0, const float* v) const {
    if (row >= B) return;
    const int qy = mode / mx, kx = mode - (mode / mx) * mx;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = c0 + q, o = col >> 1;
      Y[((((size_t)row * C + o) * mx + kx) * MY + qy) * 2 + (col & 1)] = __float2bfloat16(v[q]);
    }
  }
};

constexpr int kG4Chunk = 64;    // G4 columns per CTA: more CTAs, and shorter epilogues, at one state
struct EpiZ {    // G4 (blockIdx.z = column chunk): rows (o, kx), cols (y, re/im) -> Z1[b][o][y][kx][re/im]
  typedef NoAcc Acc;
  bf16* Z1; int Mp, mx, C;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc&, int, int, int) const {}
  __device__ void end(Acc&, int, int, int) const {}
  __device__ void chunk(Acc&, int b, int z, int row, int c0, const float* v) const {
    if (row >= C * mx) return;
    const int o = row / mx, kx = row - (row / mx) * mx;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int col = z * kG4Chunk + c0 + q, y = col >> 1;
      Z1[((((size_t)b * C + o) * Mp + y) * mx + kx) * 2 + (col & 1)] = __float2bfloat16(v[q]);
    }
  }
};

// G5: one tile = 128 pixels of one state (a row y of the network grid, or half of one at
// Mp = 256).  A1 = the inverse x-DFT matrix rows of the tile's x, B1 = the state's inverse
// y-DFT output Z1[o][y][(kx, re/im)] (24 columns, zero-padded to 32); A2 = the tile's
// activations [pixel][c], B2 = the pointwise weights W[o][c].
template <int Mp>
struct PwOps {
  const bf16 *Exi, *Z1, *act_pc, *W;
  __device__ void load(bf16* sA1, bf16* sB1, bf16* sA2, bf16* sB2) const {
    constexpr int C = 32, P = Mp * Mp, KZ = 24;
    const int tid = threadIdx.x, b = blockIdx.y;
    const int row0 = blockIdx.x * 128, y = row0 / Mp, x0 = row0 - y * Mp;
    for (int e = tid; e < 128 * 4; e += 128) {
      const int r = e >> 2, kv = e & 3;
      cp_async_16(sA1 + canon_idx(r, kv * 8, 32), Exi + (size_t)(x0 + r) * 32 + kv * 8, true);
      cp_async_16(sA2 + canon_idx(r, kv * 8, 32), act_pc + ((size_t)b * P + row0 + r) * C + kv * 8, true);
    }
    for (int e = tid; e < C * 4; e += 128) {
      const int o = e >> 2, kv = e & 3;
      const bool ok = kv * 8 < KZ;
      cp_async_16(sB1 + canon_idx(o, kv * 8, 32), ok ? Z1 + (((size_t)b * C + o) * Mp + y) * KZ + kv * 8 : Z1, ok);
      cp_async_16(sB2 + canon_idx(o, kv * 8, 32), W + (size_t)o * C + kv * 8, true);
    }
  }
};

struct EpiAct {  // G5: rows pixels, cols o -> ReLU(spectral + W v + b) into both activation layouts
  typedef NoAcc Acc;
  bf16 *act_cp, *act_pc; const float* bias; int P, C;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc&, int, int, int) const {}
  __device__ void end(Acc&, int, int, int) const {}
  __device__ void chunk(Acc&, int b, int, int p, int c0, const float* v) const {
    if (p >= P) return;
    __align__(16) bf16 h[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int o = c0 + q;
      const float x = fmaxf(v[q] + bias[o], 0.f);
      h[q] = __float2bfloat16(x);
      act_cp[((size_t)b * C + o) * P + p] = h[q];
    }
    uint4* dst = reinterpret_cast<uint4*>(act_pc + ((size_t)b * P + p) * C + c0);
    dst[0] = reinterpret_cast<const uint4*>(h)[0];
    dst[1] = reinterpret_cast<const uint4*>(h)[1];
  }
};

// Mp = 128: the two-product stage of a layer and, in the same kernel, the next layer's x-DFT
// of the tile's row (a tile is one row y of 128 pixels).  The tile's new activations go to
// shared memory as the B operand [o][x] of a third product D3[(kx, re/im)][o] = Ex act^T
// (accumulator columns 32..63), whose rows 0..23 are the x-DFT output of the row; the
// channel-major copy of the activations, which only the x-DFT read, is not written.
constexpr size_t kPwxSmem = 2 * ((size_t)2 * (128 + 32) * 32 + 128 * 128 + 32 * 128) + 64;

__global__ void __launch_bounds__(128) pino_pointwise_xdft_kernel(PwOps<128> ops, const bf16* __restrict__ Ex,
                                                                  const float* __restrict__ bias, bf16* act_pc,
                                                                  bf16* X1, int* err) {
  constexpr int Mp = 128, C = 32, P = Mp * Mp, mx = 12;
  extern __shared__ __align__(1024) unsigned char smem[];
  bf16* sA1 = reinterpret_cast<bf16*>(smem);
  bf16* sB1 = sA1 + 128 * 32;
  bf16* sA2 = sB1 + 32 * 32;
  bf16* sB2 = sA2 + 128 * 32;
  bf16* sA3 = sB2 + 32 * 32;    // x-DFT matrix rows (kx, re/im), K = x, zero below row 32
  bf16* sB3 = sA3 + 128 * 128;  // the tile's activations [o][x]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB3 + 32 * 128);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.y, y = blockIdx.x, x = tid;
  ops.load(sA1, sB1, sA2, sB2);
  for (int e = tid; e < 128 * 16; e += 128) {
    const int r = e >> 4, kv = e & 15;
    const bool ok = r < 32;
    cp_async_16(sA3 + canon_idx(r, kv * 8, 128), ok ? Ex + (size_t)r * Mp + kv * 8 : Ex, ok);
  }
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  const uint32_t tmem = umma_setup<64>(tslot, mbar);
  if (tid == 0) {
    umma_issue<32>(tmem, smem_u32(sA1), smem_u32(sB1), 32, false);
    umma_issue<32>(tmem, smem_u32(sA2), smem_u32(sB2), 32, true);
    umma_commit(mbar);
  }
  const size_t p = (size_t)y * Mp + x;
  if (umma_wait(mbar, err, 0)) {
#pragma unroll 1
    for (int c0 = 0; c0 < C; c0 += 16) {
      float v[16];
      umma_ld16(tmem, c0, v);
      __align__(16) bf16 h[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int o = c0 + q;
        h[q] = __float2bfloat16(fmaxf(v[q] + bias[o], 0.f));
        sB3[canon_idx(o, x, 128)] = h[q];
      }
      uint4* dst = reinterpret_cast<uint4*>(act_pc + ((size_t)b * P + p) * C + c0);
      dst[0] = reinterpret_cast<const uint4*>(h)[0];
      dst[1] = reinterpret_cast<const uint4*>(h)[1];
    }
  }
  // the activations, written by the threads, become the tensor cores' operand
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (tid == 0) {
    umma_issue<32>(tmem + 32, smem_u32(sA3), smem_u32(sB3), 128, false);
    umma_commit(mbar);
  }
  if (umma_wait(mbar, err, 1) && warp == 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < C; c0 += 16) {
      float v[16];
      umma_ld16(tmem + 32, c0, v);   // lane = row (kx, re/im)
      if (lane < 2 * mx) {
        const int kx = lane >> 1, ri = lane & 1;
#pragma unroll
        for (int q = 0; q < 16; ++q)
          X1[(((size_t)b * C + c0 + q) * mx + kx) * (2 * Mp) + 2 * y + ri] = __float2bfloat16(v[q]);
      }
    }
  }
  umma_teardown<64>(tmem);
}

struct ProjAcc { float s; };
struct EpiProj { // P: rows pixels, cols hidden -> w = sum_h ReLU(v + b1) w2[h] + b2
  typedef ProjAcc Acc;
  float* wout; const float* b1; const float* w2; float b2; int P;
  __device__ void prefetch(Acc&, int, int, int) const {}
  __device__ void begin(Acc& a, int, int, int) const { a.s = 0.f; }
  __device__ void chunk(Acc& a, int, int, int, int c0, const float* v) const {
#pragma unroll
    for (int q = 0; q < 16; ++q) a.s = fmaf(fmaxf(v[q] + b1[c0 + q], 0.f), w2[c0 + q], a.s);
  }
  __device__ void end(Acc& a, int b, int, int p) const {
    if (p < P) wout[(size_t)b * P + p] = a.s + b2;
  }
};

// ---------------------------------------------------------------------------------------
// CUDA-core kernels: restriction, lifting, prolongation + residual + far field (+ Parareal)
// ---------------------------------------------------------------------------------------

// bilinear sample of a node field on an Mi grid at fractional node index (ti, tj)
__device__ __forceinline__ float bilinear(const float* u, int Mi, float tx, float ty) {
  int i0 = min((int)floorf(tx), Mi - 2), j0 = min((int)floorf(ty), Mi - 2);
  i0 = max(i0, 0);
  j0 = max(j0, 0);
  const float fx = tx - i0, fy = ty - j0;
  const float* r0 = u + (size_t)j0 * Mi;
  const float* r1 = r0 + Mi;
  const float a = r0[i0] * (1.f - fx) + r0[i0 + 1] * fx;
  const float c = r1[i0] * (1.f - fx) + r1[i0 + 1] * fx;
  return a * (1.f - fy) + c * fy;
}

__global__ void pino_restrict_kernel(const PinoState* st, float* ump, int Mp) {
  const int b = blockIdx.y;
  const PinoState s = st[b];
  const size_t P = (size_t)Mp * Mp;
  const float ratio = (float)(s.M - 1) / (float)(Mp - 1);
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((unsigned)e / (unsigned)Mp), i = (int)(e - (size_t)j * Mp);
    ump[(size_t)b * P + e] = (s.M == Mp) ? s.in[e] : bilinear(s.in, s.M, i * ratio, j * ratio);
  }
}

__global__ void pino_lift_kernel(const PinoState* st, const float* ump, const float* lift_w,
                                 const float* lift_b, bf16* act_cp, bf16* act_pc, int Mp, int C,
                                 int cin) {
  const int b = blockIdx.y;
  const PinoState s = st[b];
  const size_t P = (size_t)Mp * Mp;
  const float hp = s.h * (float)(s.M - 1) / (float)(Mp - 1);   // network grid spacing
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < P; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)((unsigned)e / (unsigned)Mp), i = (int)(e - (size_t)j * Mp);
    const float a[9] = {ump[(size_t)b * P + e], i * hp, j * hp, s.tau, s.dtau, s.s1, s.s2, s.rho, s.r};
    __align__(16) bf16 h[32];
    for (int o = 0; o < C; ++o) {
      float v = lift_b[o];
      for (int c = 0; c < cin; ++c) v = fmaf(a[c], lift_w[c * C + o], v);
      h[o] = __float2bfloat16(v);
      act_cp[((size_t)b * C + o) * P + e] = h[o];
    }
    uint4* dst = reinterpret_cast<uint4*>(act_pc + ((size_t)b * P + e) * C);
    for (int q = 0; q < C / 8; ++q) dst[q] = reinterpret_cast<const uint4*>(h)[q];
  }
}

struct ApplyArgs {
  int mode;
  float* Unext;        // Parareal: u_{n+1}
  const float* Fn;     // Parareal: F(u_n)
  float* Gold;         // Parareal: G_old_n
  double* partials;    // Parareal: [blocks][2] sums of u^2 and du^2
};

// G_new = in + prolong(w) on the state grid, far field at tau + dtau; then
//   PROP: out = G_new;  INIT: u_{n+1} = G_old = G_new;  ITER: u_{n+1} = F + (G_new - G_old),
//   G_old = G_new;  ITER_SKIP: G_new = G_old (no network) and the ITER update.
// Block partial sums (FP64, fixed order) of ||u_{n+1}||^2 and ||du||^2 per block.
__global__ void pino_apply_kernel(const PinoState* st, const float* wout, int Mp, ApplyArgs aa) {
  const int b = blockIdx.y;
  const PinoState s = st[b];
  const int M = s.M;
  const size_t MM = (size_t)M * M, P = (size_t)Mp * Mp;
  const float ratio = (float)(Mp - 1) / (float)(M - 1);
  const float tau_new = s.tau + s.dtau;
  double n0 = 0.0, n1 = 0.0;
  const size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (e < MM) {
    const int j = (int)((unsigned)e / (unsigned)M), i = (int)(e - (size_t)j * M);
    float g;
    if (aa.mode == PAPPLY_ITER_SKIP) {
      g = aa.Gold[e];
    } else if (i == M - 1 || j == M - 1) {
      g = far_field(s.pf, i * s.h, j * s.h, tau_new);
    } else {
      const float w = (M == Mp) ? wout[(size_t)b * P + e] : bilinear(wout + (size_t)b * P, Mp, i * ratio, j * ratio);
      g = s.in[e] + w;
    }
    if (aa.mode == PAPPLY_PROP) {
      s.out[e] = g;
    } else if (aa.mode == PAPPLY_INIT) {
      aa.Unext[e] = g;
      aa.Gold[e] = g;
      n0 = (double)(g * g);
    } else {
      // squares in FP32 (u_new - u_old of nearby values is exact), sums in FP64
      const float unew = aa.Fn[e] + (g - aa.Gold[e]);
      const float du = unew - aa.Unext[e];
      aa.Unext[e] = unew;
      aa.Gold[e] = g;
      n0 = (double)(unew * unew);
      n1 = (double)(du * du);
    }
  }
  if (aa.mode == PAPPLY_PROP) return;
  // block reduction in a fixed order
  __shared__ double r0[32], r1[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    n0 += __shfl_xor_sync(0xffffffffu, n0, off);
    n1 += __shfl_xor_sync(0xffffffffu, n1, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { r0[warp] = n0; r1[warp] = n1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += r0[w]; s1 += r1[w]; }
    aa.partials[2 * blockIdx.x] = s0;
    aa.partials[2 * blockIdx.x + 1] = s1;
  }
}

// norms[2n] = ||u_n||^2, norms[2n+1] = ||du_n||^2 for n = n_lo..N from the block partials
// (stride pstride per slice); then delta = max_{n>n_first} ||du_n|| / max_n ||u_n||.
__global__ void pino_defect_kernel(const double* partials, int nblocks, int pstride, int n_lo,
                                   int N, int n_first, double* norms, double* defect, int iter) {
  const int lane = threadIdx.x;
  for (int n = n_lo; n <= N; ++n) {
    const double* p = partials + (size_t)n * pstride;
    double a = 0.0, c = 0.0;
    for (int k = lane; k < nblocks; k += 32) { a += p[2 * k]; c += p[2 * k + 1]; }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    if (lane == 0) { norms[2 * n] = a; norms[2 * n + 1] = iter ? c : 0.0; }
  }
  if (lane == 0 && iter) {
    double num = 0.0, den = 0.0;
    for (int n = 1; n <= N; ++n) {
      den = fmax(den, norms[2 * n]);
      if (n >= n_first + 1) num = fmax(num, norms[2 * n + 1]);
    }
    defect[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
  }
}

// ---------------------------------------------------------------------------------------
// Forward pass
// ---------------------------------------------------------------------------------------
#define BS_TRY_LAUNCH(expr) do { cudaError_t e_ = (expr); if (e_ != cudaSuccess) return cuda_error(e_, #expr); } while (0)

template <int Mp>
static int pino_network(bs_pino* net, PinoRes& R, const PinoState* st, int B, cudaStream_t s) {
  constexpr int C = 32, mx = 12, MY = 24, P = Mp * Mp;
  const int pix_blocks = (P + 255) / 256;
  pino_lift_kernel<<<dim3(pix_blocks, B), 256, 0, s>>>(st, R.ump, net->lift_w, net->lift_b,
                                                       R.act_cp, R.act_pc, Mp, C, net->cin);
  BS_CUDA_TRY(cudaGetLastError());
  const int modes = MY * mx;
  for (int l = 0; l < net->L; ++l) {
    // G1 (at Mp = 128 after the first layer it ran inside the previous layer's last stage)
    if (Mp != 128 || l == 0)
      BS_TRY_LAUNCH((launch_umma<32, Mp>(dim3(C * Mp / 128, B), GemmA{R.act_cp, (long long)C * P, Mp, C * Mp, Mp},
                                         GemmB{R.Ex, 0, 0}, EpiX1{R.X1, Mp, mx, C}, net->err, s)));
    // G2
    BS_TRY_LAUNCH((launch_umma<64, 2 * Mp>(dim3((C * mx + 127) / 128, B),
                                           GemmA{R.X1, (long long)C * mx * 2 * Mp, 2 * Mp, C * mx, 2 * Mp},
                                           GemmB{R.Ey, 0, 0}, EpiX2{R.X2, mx, MY, C, B}, net->err, s)));
    // G3 (blockIdx.y = mode)
    BS_TRY_LAUNCH((launch_umma<64, 64>(dim3(1, modes), GemmA{R.X2, (long long)B * C * 2, 64, B, 64},
                                       GemmB{net->R + (size_t)l * modes * 64 * 64, 64 * 64, 0},
                                       EpiY{R.Y, mx, MY, C, B}, net->err, s)));
    // G4 (blockIdx.z = kG4Chunk-column chunk of (y, re/im))
    BS_TRY_LAUNCH((launch_umma<kG4Chunk, 48>(dim3((C * mx + 127) / 128, B, (2 * Mp) / kG4Chunk),
                                             GemmA{R.Y, (long long)C * mx * MY * 2, MY * 2, C * mx, MY * 2},
                                             GemmB{R.Eyi, 0, kG4Chunk * 48}, EpiZ{R.Z1, Mp, mx, C}, net->err, s)));
    // G5: inverse x-DFT and the pointwise product into one accumulator (at Mp = 128, before
    // the last layer, with the next layer's x-DFT of the row)
    const PwOps<Mp> pw{R.Exi, R.Z1, R.act_pc, net->Wpw + (size_t)l * C * C};
    if constexpr (Mp == 128) {
      if (l + 1 < net->L) {
        static bool attr_set = false;
        if (!attr_set) {
          BS_CUDA_TRY(cudaFuncSetAttribute(pino_pointwise_xdft_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kPwxSmem));
          attr_set = true;
        }
        pino_pointwise_xdft_kernel<<<dim3(Mp, B), 128, kPwxSmem, s>>>(pw, R.Ex, net->pw_b + l * C, R.act_pc, R.X1,
                                                                      net->err);
        BS_CUDA_TRY(cudaGetLastError());
        continue;
      }
    }
    BS_TRY_LAUNCH((launch_umma2<32, 32, 32>(dim3(P / 128, B), pw, EpiAct{R.act_cp, R.act_pc, net->pw_b + l * C, P, C},
                                            net->err, s)));
  }
  BS_TRY_LAUNCH((launch_umma<128, 32>(dim3(P / 128, B), GemmA{R.act_pc, (long long)P * C, C, P, C},
                                      GemmB{net->W1, 0, 0}, EpiProj{R.wout, net->b1, net->w2, net->b2, P},
                                      net->err, s)));
  return BS_OK;
}

static int network_grid(int M) { return M <= 128 ? 128 : 256; }

static PinoState make_state(const ItemDesc& d, const float* in, float* out, int M, double xmax,
                            double tau, double dtau) {
  PinoState st;
  st.in = in;
  st.out = out;
  st.M = M;
  st.h = (float)(xmax / (M - 1));
  st.tau = (float)tau;
  st.dtau = (float)dtau;
  st.s1 = (float)d.s1; st.s2 = (float)d.s2; st.rho = (float)d.rho; st.r = (float)d.r;
  st.pf = make_payoff(d);
  return st;
}

// Network + residual for the states already in R.st (B of them), then the apply step.
static int pino_run(bs_pino* net, PinoRes& R, const PinoState* st, int B, int Mmax,
                    const ApplyArgs& aa, bool skip_net, cudaStream_t s) {
  const int Mp = R.Mp;
  if (!skip_net) {
    pino_restrict_kernel<<<dim3((Mp * Mp + 255) / 256, B), 256, 0, s>>>(st, R.ump, Mp);
    BS_CUDA_TRY(cudaGetLastError());
    int rc = (Mp == 128) ? pino_network<128>(net, R, st, B, s) : pino_network<256>(net, R, st, B, s);
    if (rc) return rc;
  }
  pino_apply_kernel<<<dim3((Mmax * Mmax + 255) / 256, B), 256, 0, s>>>(st, R.wout, Mp, aa);
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

int pino_check(const bs_pino* net, int M) {
  if (!net) return set_error(BS_ERR_ARG, "PINO coarse propagator needs a loaded network");
  if (net->C != 32 || net->mx != 12 || net->my != 12 || net->cin != 9 || net->H % 16 != 0 || net->H > 256)
    return set_error(BS_ERR_ARG, "PINO shape (width %d, modes %dx%d, hidden %d) not supported; "
                     "this build runs width 32, 12x12 modes, 9 inputs", net->C, net->mx, net->my, net->H);
  if (M < 8) return set_error(BS_ERR_ARG, "PINO coarse propagator: grid too small");
  return BS_OK;
}

// coarse_propagate with the PINO: one network step on one state.
int pino_propagate(bs_pino* net, const bs_grid* g, const ItemDesc& d, const float* in, float* out,
                   double tau0, double dtau, cudaStream_t s) {
  int rc = pino_check(net, g->M);
  if (rc) return rc;
  PinoRes* R;
  if ((rc = ensure_res(net, network_grid(g->M), 1, 1, &R))) return rc;
  PinoState st = make_state(d, in, out, g->M, g->xmax, tau0, dtau);
  BS_CUDA_TRY(cudaMemcpyAsync(R->st, &st, sizeof(st), cudaMemcpyHostToDevice, s));
  ApplyArgs aa = {};
  aa.mode = PAPPLY_PROP;
  return pino_run(net, *R, R->st, 1, g->M, aa, false, s);
}

// The PINO on B independent states at once (coarse_propagate_batched): one network launch
// chain per chunk of at most kPinoBatch states (the mixing GEMM holds a chunk's states in one
// 128-row tile).  A state's result does not depend on the others in its chunk: every output
// row of every GEMM is its own dot product.
constexpr int kPinoBatch = 128;
int pino_propagate_batched(bs_pino* net, const bs_grid* g, const ItemDesc* items, const float* const* in,
                           float* const* out, int B, cudaStream_t s) {
  int rc = pino_check(net, g->M);
  if (rc) return rc;
  const int chunk = B < kPinoBatch ? B : kPinoBatch;
  PinoRes* R;
  if ((rc = ensure_res(net, network_grid(g->M), chunk, chunk, &R))) return rc;
  std::vector<PinoState> sts((size_t)chunk);
  for (int b0 = 0; b0 < B; b0 += kPinoBatch) {
    const int nb = (B - b0) < kPinoBatch ? (B - b0) : kPinoBatch;
    for (int i = 0; i < nb; ++i) {
      const ItemDesc& d = items[b0 + i];
      sts[(size_t)i] = make_state(d, in[b0 + i], out[b0 + i], g->M, g->xmax, d.tau0, d.dtau);
    }
    // stream-ordered after the previous chunk's kernels, which read the descriptors
    BS_CUDA_TRY(cudaMemcpyAsync(R->st, sts.data(), (size_t)nb * sizeof(PinoState), cudaMemcpyHostToDevice, s));
    ApplyArgs aa = {};
    aa.mode = PAPPLY_PROP;
    if ((rc = pino_run(net, *R, R->st, nb, g->M, aa, false, s))) return rc;
  }
  return BS_OK;
}

// One serial Parareal sweep with the PINO as G (mode SWEEP_INIT or SWEEP_ITER), on the same
// buffers as the numerical sweep.  partials: [(N+1)][nblocks][2] doubles of workspace.
int pino_sweep(bs_pino* net, const bs_grid* g, const ItemDesc& d, const SweepArgs& a,
               double* partials, cudaStream_t s) {
  int rc = pino_check(net, g->M);
  if (rc) return rc;
  const int M = g->M;
  const size_t MM = (size_t)M * M;
  PinoRes* R;
  if ((rc = ensure_res(net, network_grid(M), 1, a.N, &R))) return rc;
  const int nblocks = (int)((MM + 255) / 256);
  const int pstride = 2 * nblocks;
  // descriptors of all slices, uploaded once (slice n reads entry n)
  std::vector<PinoState> sts((size_t)a.N);
  for (int n = 0; n < a.N; ++n)
    sts[(size_t)n] = make_state(d, a.U + (size_t)n * MM, nullptr, M, g->xmax, n * a.slice_len, a.slice_len);
  BS_CUDA_TRY(cudaMemcpyAsync(R->st, sts.data(), sts.size() * sizeof(PinoState), cudaMemcpyHostToDevice, s));
  for (int n = a.n_first; n < a.N; ++n) {
    ApplyArgs aa;
    const bool skip = (a.mode == SWEEP_ITER && n == a.n_first);
    aa.mode = a.mode == SWEEP_INIT ? PAPPLY_INIT : (skip ? PAPPLY_ITER_SKIP : PAPPLY_ITER);
    aa.Unext = a.U + (size_t)(n + 1) * MM;
    aa.Fn = a.Fb + (size_t)n * MM;
    aa.Gold = a.Gold + (size_t)n * MM;
    aa.partials = partials + (size_t)(n + 1) * pstride;
    if ((rc = pino_run(net, *R, R->st + n, 1, M, aa, skip, s))) return rc;
  }
  const int n_lo = a.mode == SWEEP_INIT ? 1 : a.n_first + 1;
  pino_defect_kernel<<<1, 32, 0, s>>>(partials, nblocks, pstride, n_lo, a.N, a.n_first, a.norms,
                                      a.defect, a.mode == SWEEP_ITER ? 1 : 0);
  BS_CUDA_TRY(cudaGetLastError());
  return BS_OK;
}

size_t pino_partials_bytes(int M, int N) {
  const size_t nblocks = ((size_t)M * M + 255) / 256;
  return (size_t)(N + 1) * nblocks * 2 * sizeof(double);
}

// kernels per network step on an M x M state: restrict, lift, 5 per layer (4 after the first
// at Mp = 128), projection, apply
int pino_launches_per_step(const bs_pino* net, int M) {
  return network_grid(M) == 128 ? 5 + 4 * net->L : 4 + 5 * net->L;
}

int pino_error_flag(const bs_pino* net, int* flag) {
  BS_CUDA_TRY(cudaMemcpy(flag, net->err, sizeof(int), cudaMemcpyDeviceToHost));
  return BS_OK;
}

}  // namespace bsp

using namespace bsp;

extern "C" int pino_load(const char* path, bs_pino** out) {
  if (out) *out = nullptr;
  if (!path || !out) return set_error(BS_ERR_ARG, "pino_load: NULL argument");
  FILE* f = fopen(path, "rb");
  if (!f) return set_error(BS_ERR_FILE, "pino_load: cannot open %s", path);
  std::vector<unsigned char> buf;
  {
    unsigned char tmp[1 << 16];
    size_t n;
    while ((n = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
    fclose(f);
  }
  if (buf.size() < 40 || std::memcmp(buf.data(), "BSPINO01", 8) != 0)
    return set_error(BS_ERR_FILE, "pino_load: %s is not a PINO weight file", path);
  int32_t hdr[8];
  std::memcpy(hdr, buf.data() + 8, sizeof(hdr));
  const int cin = hdr[0], C = hdr[1], mx = hdr[2], my = hdr[3], L = hdr[4], H = hdr[5];
  if (cin < 1 || C < 1 || mx < 1 || my < 1 || L < 1 || H < 1 || cin > 64 || C > 256 || L > 64 || H > 4096)
    return set_error(BS_ERR_FILE, "pino_load: %s: implausible header", path);
  const size_t MYx = (size_t)2 * my * mx;
  const size_t nfloat = (size_t)cin * C + C + 2 * (size_t)L * MYx * C * C + (size_t)L * C * C +
                        (size_t)L * C + (size_t)C * H + H + H + 1;
  if (buf.size() != 40 + 4 * nfloat)
    return set_error(BS_ERR_FILE, "pino_load: %s: size %zu, expected %zu", path, buf.size(), 40 + 4 * nfloat);
  const float* fp = reinterpret_cast<const float*>(buf.data() + 40);
  auto take = [&](size_t n) { std::vector<float> v(fp, fp + n); fp += n; return v; };
  std::vector<float> lift_w = take((size_t)cin * C), lift_b = take(C);
  std::vector<float> sre = take((size_t)L * MYx * C * C), sim = take((size_t)L * MYx * C * C);
  std::vector<float> pw_w = take((size_t)L * C * C), pw_b = take((size_t)L * C);
  std::vector<float> p1w = take((size_t)C * H), p1b = take(H), p2w = take(H), p2b = take(1);

  bs_pino* net = new bs_pino();
  std::memset(net, 0, sizeof(*net));
  net->cin = cin; net->C = C; net->mx = mx; net->my = my; net->L = L; net->H = H; net->b2 = p2b[0];
  // complex mode matrices in real 2x2 block form: rows (o, re/im), columns (c, re/im)
  std::vector<bf16> R((size_t)L * MYx * 2 * C * 2 * C);
  for (int l = 0; l < L; ++l)
    for (size_t m = 0; m < MYx; ++m)
      for (int c = 0; c < C; ++c)
        for (int o = 0; o < C; ++o) {
          const size_t src = (((size_t)l * MYx + m) * C + c) * C + o;
          const float re = sre[src], im = sim[src];
          bf16* blk = R.data() + ((size_t)l * MYx + m) * (2 * C) * (2 * C);
          blk[(2 * o) * (2 * C) + 2 * c] = __float2bfloat16(re);
          blk[(2 * o) * (2 * C) + 2 * c + 1] = __float2bfloat16(-im);
          blk[(2 * o + 1) * (2 * C) + 2 * c] = __float2bfloat16(im);
          blk[(2 * o + 1) * (2 * C) + 2 * c + 1] = __float2bfloat16(re);
        }
  std::vector<bf16> Wpw((size_t)L * C * C), W1((size_t)H * C);
  for (int l = 0; l < L; ++l)
    for (int c = 0; c < C; ++c)
      for (int o = 0; o < C; ++o) Wpw[((size_t)l * C + o) * C + c] = __float2bfloat16(pw_w[((size_t)l * C + c) * C + o]);
  for (int c = 0; c < C; ++c)
    for (int h = 0; h < H; ++h) W1[(size_t)h * C + c] = __float2bfloat16(p1w[(size_t)c * H + h]);
  int rc;
  if ((rc = upload(&net->lift_w, lift_w)) || (rc = upload(&net->lift_b, lift_b)) ||
      (rc = upload(&net->R, R)) || (rc = upload(&net->Wpw, Wpw)) || (rc = upload(&net->pw_b, pw_b)) ||
      (rc = upload(&net->W1, W1)) || (rc = upload(&net->b1, p1b)) || (rc = upload(&net->w2, p2w)) ||
      (rc = dev_alloc((void**)&net->err, sizeof(int)))) {
    pino_destroy(net);
    return rc;
  }
  cudaMemset(net->err, 0, sizeof(int));
  *out = net;
  return BS_OK;
}

extern "C" int pino_destroy(bs_pino* net) {
  if (!net) return BS_OK;
  void* ptrs[] = {net->lift_w, net->lift_b, net->R, net->Wpw, net->pw_b, net->W1, net->b1, net->w2, net->err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_res(net->res[0]);
  free_res(net->res[1]);
  delete net;
  return BS_OK;
}
