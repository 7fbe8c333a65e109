// les_unet.cu -- the learned Poisson warm start: a 3-level 3-D U-Net trained
// and evaluated with this library's own BF16 tensor-core kernels (FP32
// accumulation).  Not in the paper; it predicts the first guess psi_0 of the
// pressure-correction solve (Sec. 2.4) from its right-hand side b:
//
//   x0 = b / s, s = rms(b);  e1 = B(x0; 1->16);  e2 = B(pool e1; 16->32);
//   e3 = B(pool e2; 32->64);  g2 = B([up e3, e2]; 96->32);
//   g1 = B([up g2, e1]; 48->16);  y = conv1(g1; 16->1);  psi_0 = s (y - mean y)
//
// with B(.; a->c) two 3x3x3 periodic convolutions each followed by a leaky
// ReLU (slope 0.1), pool a 2x2x2 mean, up nearest-neighbour doubling and
// [.,.] channel concatenation.  Weights travel as one flat FP32 vector, layer
// by layer, W[cout][cin][kz][ky][kx] then bias[cout].
//
// Kernels: activations are channels-last BF16 ([batch][z][y][x][c], c
// padded to a multiple of 16).  A convolution is an implicit GEMM on the
// tensor cores -- rows are 16 voxels, K runs over (tap, 16-channel slab), N
// over output channels -- issued as mma.sync m16n8k16 BF16 -> FP32 with the
// bias and activation fused into the epilogue.  The input-gradient pass is
// the same kernel on flipped, transposed weights; the weight gradient is a
// second tensor-core GEMM over voxel chunks whose FP32 partials are summed in
// chunk order (deterministic).  Adam keeps FP32 master weights.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "les_internal.h"

namespace les {
namespace {

using bf16 = __nv_bfloat16;
constexpr float kLeak = 0.1f;

struct LayerDef {
  const char* name;
  int cin, cout, k;
};
constexpr LayerDef kLayers[] = {{"enc1a", 1, 16, 3},  {"enc1b", 16, 16, 3}, {"enc2a", 16, 32, 3},
                                {"enc2b", 32, 32, 3}, {"enc3a", 32, 64, 3}, {"enc3b", 64, 64, 3},
                                {"dec2a", 96, 32, 3}, {"dec2b", 32, 32, 3}, {"dec1a", 48, 16, 3},
                                {"dec1b", 16, 16, 3}, {"head", 16, 1, 1}};
constexpr int kNL = 11;
enum { L_E1A, L_E1B, L_E2A, L_E2B, L_E3A, L_E3B, L_D2A, L_D2B, L_D1A, L_D1B, L_HEAD };

__host__ __device__ inline int pad16(int c) { return (c + 15) / 16 * 16; }
__host__ __device__ inline int pad8(int c) { return (c + 7) / 8 * 8; }

// ---- tensor-core primitive ----------------------------------------------------
__device__ __forceinline__ void mma_bf16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ unsigned ld32(const bf16* p) { return *reinterpret_cast<const unsigned*>(p); }
__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}
__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// voxel index of the tap neighbour of voxel v (cubic grid n, periodic)
__device__ __forceinline__ int nbr(int v, int n, int dz, int dy, int dx) {
  const int x = v % n, y = (v / n) % n, zb = v / (n * n);
  const int z = zb % n, b = zb / n;
  return ((b * n + wrapn(z + dz, n)) * n + wrapn(y + dy, n)) * n + wrapn(x + dx, n);
}

// ---- convolution as an implicit GEMM --------------------------------------------
struct ConvArgs {
  const bf16* in0;
  int c0;  // channels of in0 (multiple of 16)
  const bf16* in1;
  int c1;  // channels of in1 (0 if absent)
  const bf16* w;  // [taps][cout][cin] with cin = c0 + c1
  const float* bias;
  void* out0;
  int oc0;
  void* out1;
  int oc1;
  int n, nvox, k;
  int act;
};

// 4 warps x 16 voxels per block; NF output-channel fragments of 8
template <int NF, bool OUT_F32>
__global__ void __launch_bounds__(128) k_conv(ConvArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int v0 = (blockIdx.x * 4 + warp) * 16;
  if (v0 >= a.nvox) return;
  const int cin = a.c0 + a.c1;
  const int r = a.k / 2;
  const int rowA = v0 + gid, rowB = v0 + gid + 8;
  const bool okA = rowA < a.nvox, okB = rowB < a.nvox;
  float acc[NF][4];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = 0.f;
  const int ntap = a.k * a.k * a.k;
  for (int t = 0; t < ntap; ++t) {
    const int dz = t / (a.k * a.k) - r, dy = (t / a.k) % a.k - r, dx = t % a.k - r;
    const int na = nbr(okA ? rowA : v0, a.n, dz, dy, dx), nb = nbr(okB ? rowB : v0, a.n, dz, dy, dx);
    const bf16* wt = a.w + (size_t)t * (NF * 8) * cin;
    for (int kc = 0; kc < cin; kc += 16) {
      const bf16* src;
      int cs, cc;
      if (kc < a.c0) {
        src = a.in0;
        cs = a.c0;
        cc = kc;
      } else {
        src = a.in1;
        cs = a.c1;
        cc = kc - a.c0;
      }
      const bf16* pa = src + (size_t)na * cs + cc + tig * 2;
      const bf16* pb = src + (size_t)nb * cs + cc + tig * 2;
      const unsigned a0 = okA ? ld32(pa) : 0u, a1 = okB ? ld32(pb) : 0u;
      const unsigned a2 = okA ? ld32(pa + 8) : 0u, a3 = okB ? ld32(pb + 8) : 0u;
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const bf16* pw = wt + (size_t)(f * 8 + gid) * cin + kc + tig * 2;
        mma_bf16(acc[f], a0, a1, a2, a3, ld32(pw), ld32(pw + 8));
      }
    }
  }
  // epilogue: bias, activation, split store
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int co = f * 8 + tig * 2;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int v = h ? rowB : rowA;
      if (v >= a.nvox) continue;
      float x0 = acc[f][2 * h], x1 = acc[f][2 * h + 1];
      if (a.bias) {
        x0 += a.bias[co];
        x1 += a.bias[co + 1];
      }
      if (a.act) {
        x0 = x0 > 0.f ? x0 : kLeak * x0;
        x1 = x1 > 0.f ? x1 : kLeak * x1;
      }
      if (co < a.oc0) {
        if (OUT_F32) {
          float* o = reinterpret_cast<float*>(a.out0) + (size_t)v * a.oc0 + co;
          *reinterpret_cast<float2*>(o) = make_float2(x0, x1);
        } else {
          bf16* o = reinterpret_cast<bf16*>(a.out0) + (size_t)v * a.oc0 + co;
          *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(x0, x1);
        }
      } else if (co - a.oc0 < a.oc1) {
        bf16* o = reinterpret_cast<bf16*>(a.out1) + (size_t)v * a.oc1 + (co - a.oc0);
        *reinterpret_cast<__nv_bfloat162*>(o) = __floats2bfloat162_rn(x0, x1);
      }
    }
  }
}

// ---- weight gradient: gW[t][co][ci] = sum_v g[v][co] in[nbr(v, t)][ci] ----------
struct WgradArgs {
  const bf16* g;  // [nvox][gstride]
  int gstride;
  int cout;       // channels of g that take part (the rest read as 0)
  const bf16* in0;
  int c0;
  const bf16* in1;
  int c1;
  float* part;  // [nchunk][taps][cout16][cin]
  int n, nvox, k, chunk;
};

// one warp per (tap, 16 output channels, voxel chunk); NF = cin / 8 fragments
template <int NF>
__global__ void __launch_bounds__(32) k_wgrad(WgradArgs a) {
  const int lane = threadIdx.x, gid = lane >> 2, tig = lane & 3;
  const int t = blockIdx.x, cob = blockIdx.y, ch = blockIdx.z;
  const int cin = a.c0 + a.c1;
  const int r = a.k / 2;
  const int dz = t / (a.k * a.k) - r, dy = (t / a.k) % a.k - r, dx = t % a.k - r;
  const int co_a = cob * 16 + gid, co_b = co_a + 8;
  const bool ok_a = co_a < a.cout, ok_b = co_b < a.cout;
  const bf16 zero = __float2bfloat16(0.f);
  float acc[NF][4];
#pragma unroll
  for (int f = 0; f < NF; ++f) acc[f][0] = acc[f][1] = acc[f][2] = acc[f][3] = 0.f;
  const int vend = min(a.nvox, (ch + 1) * a.chunk);
  for (int v0 = ch * a.chunk; v0 < vend; v0 += 16) {
    const int va = v0 + tig * 2, vb = va + 8;  // K index (voxel) of this thread's fragment entries
    // A (16 co x 16 voxels): A[m][k] = g[v0 + k][co0 + m]
    auto gv = [&](int v, int co, bool ok) { return ok && v < vend ? a.g[(size_t)v * a.gstride + co] : zero; };
    const unsigned a0 = pack2(gv(va, co_a, ok_a), gv(va + 1, co_a, ok_a));
    const unsigned a1 = pack2(gv(va, co_b, ok_b), gv(va + 1, co_b, ok_b));
    const unsigned a2 = pack2(gv(vb, co_a, ok_a), gv(vb + 1, co_a, ok_a));
    const unsigned a3 = pack2(gv(vb, co_b, ok_b), gv(vb + 1, co_b, ok_b));
    const bool k0 = va < vend, k1 = va + 1 < vend, k2 = vb < vend, k3 = vb + 1 < vend;
    const int n0 = nbr(k0 ? va : v0, a.n, dz, dy, dx), n1 = nbr(k1 ? va + 1 : v0, a.n, dz, dy, dx);
    const int n2 = nbr(k2 ? vb : v0, a.n, dz, dy, dx), n3 = nbr(k3 ? vb + 1 : v0, a.n, dz, dy, dx);
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const int ci = f * 8 + gid;
      const bf16* src;
      int cs, cc;
      if (ci < a.c0) {
        src = a.in0;
        cs = a.c0;
        cc = ci;
      } else {
        src = a.in1;
        cs = a.c1;
        cc = ci - a.c0;
      }
      // B (16 voxels x 8 ci): B[k][n] = in[nbr(v0 + k)][ci0 + n]
      const unsigned b0 = pack2(k0 ? src[(size_t)n0 * cs + cc] : zero, k1 ? src[(size_t)n1 * cs + cc] : zero);
      const unsigned b1 = pack2(k2 ? src[(size_t)n2 * cs + cc] : zero, k3 ? src[(size_t)n3 * cs + cc] : zero);
      mma_bf16(acc[f], a0, a1, a2, a3, b0, b1);
    }
  }
  const int ntap = a.k * a.k * a.k;
  const int co16 = (a.cout + 15) / 16 * 16;
  float* base = a.part + (((size_t)ch * ntap + t) * co16) * cin;
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const int ci = f * 8 + tig * 2;
    base[(size_t)co_a * cin + ci] = acc[f][0];
    base[(size_t)co_a * cin + ci + 1] = acc[f][1];
    base[(size_t)co_b * cin + ci] = acc[f][2];
    base[(size_t)co_b * cin + ci + 1] = acc[f][3];
  }
}

// sum the chunk partials (chunk order) into the flat FP32 gradient
// (layout W[co][ci][tap] of the real, unpadded channels)
__global__ void k_wgrad_reduce(const float* part, int nchunk, int ntap, int co16, int cin_pad, int cout,
                               int cin, float* gflat) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int total = cout * cin * ntap;
  if (idx >= total) return;
  const int t = idx % ntap, ci = (idx / ntap) % cin, co = idx / (ntap * cin);
  float s = 0.f;
  for (int c = 0; c < nchunk; ++c) s += part[(((size_t)c * ntap + t) * co16 + co) * cin_pad + ci];
  gflat[idx] = s;
}

// bias gradient: sum over voxels of g[v][co] (two passes, fixed order)
__global__ void k_bias_partial(const bf16* g, int gstride, int cout_pad, int nvox, int chunk, float* part) {
  const int co = threadIdx.x, ch = blockIdx.x;
  if (co >= cout_pad) return;
  float s = 0.f;
  const int vend = min(nvox, (ch + 1) * chunk);
  for (int v = ch * chunk; v < vend; ++v) s += __bfloat162float(g[(size_t)v * gstride + co]);
  part[(size_t)ch * cout_pad + co] = s;
}
__global__ void k_bias_reduce(const float* part, int nchunk, int cout_pad, int cout, float* gb) {
  const int co = threadIdx.x;
  if (co >= cout) return;
  float s = 0.f;
  for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * cout_pad + co];
  gb[co] = s;
}

// ---- elementwise and resampling ---------------------------------------------------
__global__ void k_pool(const bf16* in, int c, int n, int batch, bf16* out) {
  const int m = n / 2;
  const long long total = (long long)batch * m * m * m * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long v = i / c;
    const int x = (int)(v % m), y = (int)((v / m) % m), z = (int)((v / ((long long)m * m)) % m);
    const int b = (int)(v / ((long long)m * m * m));
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
      s += __bfloat162float(in[((((size_t)b * n + zz) * n + yy) * n + xx) * c + ch]);
    }
    out[i] = __float2bfloat16(s * 0.125f);
  }
}
// gradient of pool: g_in[fine] (+)= g_out[coarse] / 8
__global__ void k_pool_bwd(const bf16* gout, int c, int n, int batch, bf16* gin, int accumulate) {
  const int m = n / 2;
  const long long total = (long long)batch * n * n * n * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long v = i / c;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)((v / ((long long)n * n)) % n);
    const int b = (int)(v / ((long long)n * n * n));
    float g = __bfloat162float(gout[((((size_t)b * m + z / 2) * m + y / 2) * m + x / 2) * c + ch]) * 0.125f;
    if (accumulate) g += __bfloat162float(gin[i]);
    gin[i] = __float2bfloat16(g);
  }
}
// nearest-neighbour doubling from an m-grid to n = 2m
__global__ void k_up(const bf16* in, int c, int m, int batch, bf16* out) {
  const int n = 2 * m;
  const long long total = (long long)batch * n * n * n * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long v = i / c;
    const int x = (int)(v % n), y = (int)((v / n) % n), z = (int)((v / ((long long)n * n)) % n);
    const int b = (int)(v / ((long long)n * n * n));
    out[i] = in[((((size_t)b * m + z / 2) * m + y / 2) * m + x / 2) * c + ch];
  }
}
// gradient of up: sum of the 8 fine children
__global__ void k_up_bwd(const bf16* gout, int c, int m, int batch, bf16* gin) {
  const int n = 2 * m;
  const long long total = (long long)batch * m * m * m * c;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(i % c);
    long long v = i / c;
    const int x = (int)(v % m), y = (int)((v / m) % m), z = (int)((v / ((long long)m * m)) % m);
    const int b = (int)(v / ((long long)m * m * m));
    float s = 0.f;
    for (int q = 0; q < 8; ++q) {
      const int xx = 2 * x + (q & 1), yy = 2 * y + ((q >> 1) & 1), zz = 2 * z + (q >> 2);
      s += __bfloat162float(gout[((((size_t)b * n + zz) * n + yy) * n + xx) * c + ch]);
    }
    gin[i] = __float2bfloat16(s);
  }
}
// leaky ReLU backward from the post-activation (same sign as the pre-activation)
__global__ void k_act_bwd(const bf16* post, const bf16* g, long long total, bf16* out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float gv = __bfloat162float(g[i]);
    out[i] = __float2bfloat16(__bfloat162float(post[i]) > 0.f ? gv : kLeak * gv);
  }
}

// per-sample FP64 sum of squares of b (n3 values per sample)
template <typename T>
__global__ void k_sumsq(const T* b, long long n3, double* out) {
  __shared__ double sh[32];
  const int s = blockIdx.y;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
    const double x = (double)b[(size_t)s * n3 + i];
    acc += x * x;
  }
  const double r = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) out[(size_t)s * gridDim.x + blockIdx.x] = r;
}
// s = sqrt(mean b^2) per sample from the block partials
__global__ void k_scale(const double* part, int nblk, long long n3, int batch, double* scale) {
  const int s = threadIdx.x;
  if (s >= batch) return;
  double acc = 0.0;
  for (int q = 0; q < nblk; ++q) acc += part[(size_t)s * nblk + q];
  scale[s] = sqrt(acc / (double)n3);
}
// x0[v][0] = b / s, other 15 channels 0; optional normalised target t = psi / s
template <typename T>
__global__ void k_pack(const T* b, const T* psi, long long n3, int batch, const double* scale, double out_scale,
                       bf16* x0, float* tgt) {
  const long long total = (long long)batch * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / n3);
    const double sc = scale[s];
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    __nv_bfloat162 lo = __floats2bfloat162_rn((float)((double)b[i] * inv), 0.f);
    __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(x0 + (size_t)i * 16);
    o[0] = lo;
#pragma unroll
    for (int q = 1; q < 8; ++q) o[q] = z;
    if (tgt) tgt[i] = (float)((double)psi[i] * inv / out_scale);
  }
}
// MSE over batch x n3 of y (channel 0 of [.][8] FP32) vs t; gy = 2 (y - t) / count
// in channel 0 of a 16-channel BF16 gradient
__global__ void k_loss(const float* y, const float* t, long long total, bf16* gy, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const float inv = 2.f / (float)total;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[(size_t)i * 8] - t[i];
    acc += (double)d * d;
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(gy + (size_t)i * 16);
    o[0] = __floats2bfloat162_rn(d * inv, 0.f);
    const __nv_bfloat162 z = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int q = 1; q < 8; ++q) o[q] = z;
  }
  const double r = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}
// Energy norm of the error on the periodic n^3 grid (unit spacing) over
// batch samples: loss = sum d (6 d - sum of the six neighbours) / count,
// d = y - t; gy = 2 (6 d - sum of the six neighbours) / count in channel 0.
__global__ void k_loss_energy(const float* y, const float* t, int n, long long total, bf16* gy, double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  const float inv = 2.f / (float)total;
  const long long n3 = (long long)n * n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long s0 = (i / n3) * n3;
    const int v = (int)(i - s0);
    const int x = v % n, yy = (v / n) % n, z = v / (n * n);
    auto d = [&](int xx, int yv, int zz) {
      const long long q = s0 + ((long long)zz * n + yv) * n + xx;
      return y[(size_t)q * 8] - t[q];
    };
    const float d0 = d(x, yy, z);
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    const int ym = yy == 0 ? n - 1 : yy - 1, yp = yy == n - 1 ? 0 : yy + 1;
    const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
    const float ld = 6.f * d0 - (d(xm, yy, z) + d(xp, yy, z)) - (d(x, ym, z) + d(x, yp, z)) -
                     (d(x, yy, zm) + d(x, yy, zp));
    acc += (double)d0 * ld;
    __nv_bfloat162* o = reinterpret_cast<__nv_bfloat162*>(gy + (size_t)i * 16);
    o[0] = __floats2bfloat162_rn(ld * inv, 0.f);
    const __nv_bfloat162 zr = __floats2bfloat162_rn(0.f, 0.f);
#pragma unroll
    for (int q = 1; q < 8; ++q) o[q] = zr;
  }
  const double r = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = r;
}
__global__ void k_sum_part(const double* part, int n, double* out) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
  const double r = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) *out = r;
}
// per-sample mean of y (channel 0)
__global__ void k_ymean(const float* y, long long n3, double* out) {
  __shared__ double sh[32];
  const int s = blockIdx.x;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n3; i += blockDim.x) acc += (double)y[((size_t)s * n3 + i) * 8];
  const double r = block_reduce<false>(acc, sh);
  if (threadIdx.x == 0) out[s] = r / (double)n3;
}
// psi_0 = s (y - mean y)
template <typename T>
__global__ void k_unpack(const float* y, long long n3, int batch, const double* scale, double out_scale,
                         const double* ymean, T* psi) {
  const long long total = (long long)batch * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(i / n3);
    psi[i] = (T)(scale[s] * out_scale * ((double)y[(size_t)i * 8] - ymean[s]));
  }
}

// master FP32 (flat) -> forward BF16 [tap][co_pad8][ci_pad16] and backward
// BF16 [flipped tap][ci_pad16][co_pad8 -> padded to 16] weights, FP32 bias
__global__ void k_weights(const float* flat, int cin, int cout, int k, int cinp, int coutp, int coutp16,
                          bf16* wf, bf16* wb, float* bias) {
  const int ntap = k * k * k;
  const int total = ntap * coutp16 * cinp;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int ci = i % cinp, co = (i / cinp) % coutp16, t = i / (cinp * coutp16);
    const float w = (co < cout && ci < cin) ? flat[((size_t)co * cin + ci) * ntap + t] : 0.f;
    if (co < coutp) wf[((size_t)t * coutp + co) * cinp + ci] = __float2bfloat16(w);
    // backward data: out channel = ci, in channel = co, tap flipped
    wb[((size_t)(ntap - 1 - t) * cinp + ci) * coutp16 + co] = __float2bfloat16(w);
  }
  if (blockIdx.x == 0)
    for (int co = threadIdx.x; co < coutp; co += blockDim.x)
      bias[co] = co < cout ? flat[(size_t)cout * cin * ntap + co] : 0.f;
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace
}  // namespace les

// ============================================================================
// host side
// ============================================================================
using namespace les;

struct les_unet {
  int n = 0, batch = 0;
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  int nsm = 148;
  size_t nparams = 0;
  size_t woff[kNL] = {};  // flat offsets of each layer's W (bias follows)
  // device buffers
  float *master = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
  bf16* wf[kNL] = {};
  bf16* wb[kNL] = {};
  float* bias[kNL] = {};
  bf16 *x0, *a1a, *e1, *p1, *a2a, *e2, *p2, *a3a, *e3, *u3, *a4a, *g2, *u2, *a5a, *g1;
  float *y, *tgt;
  bf16 *G0, *G1, *G2, *G3, *G4;  // gradient scratch (largest level, 48 channels)
  float* wpart = nullptr;
  size_t wpart_floats = 0;
  double *scale, *ymean, *dpart, *loss;
  int step = 0;
  int loss_kind = 0;       // 0 mean squared error, 1 energy norm of the error
  double out_scale = 1.0;  // psi_0 = s * out_scale * (y - mean y)
  std::string err;
  Profiler* prof = nullptr;
};

namespace {

struct Carve {
  char* base;
  size_t off = 0;
  bool dry;
  template <typename P>
  P* take(size_t bytes) {
    off = (off + 255) / 256 * 256;
    P* p = dry ? nullptr : reinterpret_cast<P*>(base + off);
    off += bytes;
    return p;
  }
};

size_t layout(les_unet* u, char* base, bool dry) {
  Carve c{base, 0, dry};
  const size_t n3 = (size_t)u->n * u->n * u->n, B = (size_t)u->batch;
  const size_t v1 = B * n3, v2 = v1 / 8, v3 = v2 / 8;
  size_t np = 0;
  for (int l = 0; l < kNL; ++l) {
    u->woff[l] = np;
    np += (size_t)kLayers[l].cout * kLayers[l].cin * kLayers[l].k * kLayers[l].k * kLayers[l].k + kLayers[l].cout;
  }
  u->nparams = np;
  u->master = c.take<float>(np * 4);
  u->grad = c.take<float>(np * 4);
  u->m1 = c.take<float>(np * 4);
  u->m2 = c.take<float>(np * 4);
  size_t maxpart = 0;
  for (int l = 0; l < kNL; ++l) {
    const LayerDef& L = kLayers[l];
    const int nt = L.k * L.k * L.k, cinp = pad16(L.cin), cop = pad8(L.cout), cop16 = pad16(L.cout);
    u->wf[l] = c.take<bf16>((size_t)nt * cop * cinp * 2);
    u->wb[l] = c.take<bf16>((size_t)nt * cinp * cop16 * 2);
    u->bias[l] = c.take<float>((size_t)cop * 4);
    const size_t nv = (l <= L_E1B || l >= L_D1A) ? v1 : ((l <= L_E2B || l >= L_D2A) ? v2 : v3);
    const size_t nch = (nv + 4095) / 4096;
    maxpart = std::max(maxpart, nch * nt * (size_t)cop16 * cinp);
  }
  u->x0 = c.take<bf16>(v1 * 16 * 2);
  u->a1a = c.take<bf16>(v1 * 16 * 2);
  u->e1 = c.take<bf16>(v1 * 16 * 2);
  u->p1 = c.take<bf16>(v2 * 16 * 2);
  u->a2a = c.take<bf16>(v2 * 32 * 2);
  u->e2 = c.take<bf16>(v2 * 32 * 2);
  u->p2 = c.take<bf16>(v3 * 32 * 2);
  u->a3a = c.take<bf16>(v3 * 64 * 2);
  u->e3 = c.take<bf16>(v3 * 64 * 2);
  u->u3 = c.take<bf16>(v2 * 64 * 2);
  u->a4a = c.take<bf16>(v2 * 32 * 2);
  u->g2 = c.take<bf16>(v2 * 32 * 2);
  u->u2 = c.take<bf16>(v1 * 32 * 2);
  u->a5a = c.take<bf16>(v1 * 16 * 2);
  u->g1 = c.take<bf16>(v1 * 16 * 2);
  u->y = c.take<float>(v1 * 8 * 4);
  u->tgt = c.take<float>(v1 * 4);
  for (bf16** g : {&u->G0, &u->G1, &u->G2, &u->G3, &u->G4}) *g = c.take<bf16>(v1 * 48 * 2);
  u->wpart_floats = maxpart;
  u->wpart = c.take<float>(maxpart * 4);
  u->scale = c.take<double>(B * 8);
  u->ymean = c.take<double>(B * 8);
  u->dpart = c.take<double>(8192 * 8);
  u->loss = c.take<double>(8);
  return c.off + 256;
}

int unet_fail(les_unet* u, cudaError_t e, const char* where) {
  u->err = std::string(where) + ": " + cudaGetErrorString(e);
  return LES_ERR_CUDA;
}

unsigned eblocks(long long total) { return (unsigned)std::min<long long>((total + 255) / 256, 8192); }

template <int NF>
void launch_conv_nf(const ConvArgs& a, bool f32, cudaStream_t st) {
  const unsigned blocks = (unsigned)((a.nvox / 16 + 3) / 4);
  if (f32) k_conv<NF, true><<<blocks, 128, 0, st>>>(a);
  else k_conv<NF, false><<<blocks, 128, 0, st>>>(a);
}

// conv over nvox voxels: in = [in0 (c0), in1 (c1)] -> out = [out0 (oc0), out1 (oc1)]
cudaError_t conv(les_unet* u, int level_n, int nvox, const bf16* in0, int c0, const bf16* in1, int c1, const bf16* w,
                 const float* bias, int k, void* out0, int oc0, void* out1, int oc1, bool act, bool f32) {
  ConvArgs a{in0, c0, in1, c1, w, bias, out0, oc0, out1, oc1, level_n, nvox, k, act ? 1 : 0};
  const int nf = (oc0 + oc1) / 8;
  ProfScope ps(u->prof, KI_UNET_CONV, u->st);
  switch (nf) {
    case 1: launch_conv_nf<1>(a, f32, u->st); break;
    case 2: launch_conv_nf<2>(a, f32, u->st); break;
    case 4: launch_conv_nf<4>(a, f32, u->st); break;
    case 6: launch_conv_nf<6>(a, f32, u->st); break;
    case 8: launch_conv_nf<8>(a, f32, u->st); break;
    case 12: launch_conv_nf<12>(a, f32, u->st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int NF>
void launch_wgrad_nf(const WgradArgs& a, dim3 grid, cudaStream_t st) {
  k_wgrad<NF><<<grid, 32, 0, st>>>(a);
}

// weight + bias gradient of layer l given g (gradient at its pre-activation)
cudaError_t wgrad(les_unet* u, int l, int level_n, int nvox, const bf16* g, int gstride, const bf16* in0, int c0,
                  const bf16* in1, int c1) {
  const LayerDef& L = kLayers[l];
  const int nt = L.k * L.k * L.k, cop = pad8(L.cout), cop16 = pad16(L.cout), cin = c0 + c1;
  const int chunk = 4096;
  const int nch = (nvox + chunk - 1) / chunk;
  WgradArgs a{g, gstride, cop, in0, c0, in1, c1, u->wpart, level_n, nvox, L.k, chunk};
  dim3 grid(nt, cop16 / 16, nch);
  {
    ProfScope ps(u->prof, KI_UNET_WGRAD, u->st);
    switch (cin / 8) {
      case 2: launch_wgrad_nf<2>(a, grid, u->st); break;
      case 4: launch_wgrad_nf<4>(a, grid, u->st); break;
      case 6: launch_wgrad_nf<6>(a, grid, u->st); break;
      case 8: launch_wgrad_nf<8>(a, grid, u->st); break;
      case 12: launch_wgrad_nf<12>(a, grid, u->st); break;
      default: return cudaErrorInvalidValue;
    }
  }
  const int total = L.cout * L.cin * nt;
  k_wgrad_reduce<<<(total + 255) / 256, 256, 0, u->st>>>(u->wpart, nch, nt, cop16, cin, L.cout, L.cin,
                                                         u->grad + u->woff[l]);
  const int bchunk = 2048, nb = (nvox + bchunk - 1) / bchunk;
  float* bpart = u->wpart;  // free again after the reduce (stream order)
  k_bias_partial<<<nb, std::max(32, cop), 0, u->st>>>(g, gstride, cop, nvox, bchunk, bpart);
  k_bias_reduce<<<1, std::max(32, cop), 0, u->st>>>(bpart, nb, cop, L.cout,
                                                    u->grad + u->woff[l] + (size_t)L.cout * L.cin * nt);
  return cudaGetLastError();
}

cudaError_t refresh_weights(les_unet* u) {
  for (int l = 0; l < kNL; ++l) {
    const LayerDef& L = kLayers[l];
    const int nt = L.k * L.k * L.k;
    const int total = nt * pad16(L.cout) * pad16(L.cin);
    k_weights<<<(total + 255) / 256, 256, 0, u->st>>>(u->master + u->woff[l], L.cin, L.cout, L.k, pad16(L.cin),
                                                      pad8(L.cout), pad16(L.cout), u->wf[l], u->wb[l], u->bias[l]);
  }
  return cudaGetLastError();
}

// forward pass on the packed input x0 (batch b); y receives the head output
cudaError_t forward(les_unet* u, int b) {
  const int n1 = u->n, n2 = n1 / 2, n3 = n2 / 2;
  const int v1 = b * n1 * n1 * n1, v2 = v1 / 8, v3 = v2 / 8;
  cudaError_t e;
#define CK(x)                               \
  if ((e = (x)) != cudaSuccess) return e;
  CK(conv(u, n1, v1, u->x0, 16, nullptr, 0, u->wf[L_E1A], u->bias[L_E1A], 3, u->a1a, 16, nullptr, 0, true, false));
  CK(conv(u, n1, v1, u->a1a, 16, nullptr, 0, u->wf[L_E1B], u->bias[L_E1B], 3, u->e1, 16, nullptr, 0, true, false));
  k_pool<<<eblocks((long long)v2 * 16), 256, 0, u->st>>>(u->e1, 16, n1, b, u->p1);
  CK(conv(u, n2, v2, u->p1, 16, nullptr, 0, u->wf[L_E2A], u->bias[L_E2A], 3, u->a2a, 32, nullptr, 0, true, false));
  CK(conv(u, n2, v2, u->a2a, 32, nullptr, 0, u->wf[L_E2B], u->bias[L_E2B], 3, u->e2, 32, nullptr, 0, true, false));
  k_pool<<<eblocks((long long)v3 * 32), 256, 0, u->st>>>(u->e2, 32, n2, b, u->p2);
  CK(conv(u, n3, v3, u->p2, 32, nullptr, 0, u->wf[L_E3A], u->bias[L_E3A], 3, u->a3a, 64, nullptr, 0, true, false));
  CK(conv(u, n3, v3, u->a3a, 64, nullptr, 0, u->wf[L_E3B], u->bias[L_E3B], 3, u->e3, 64, nullptr, 0, true, false));
  k_up<<<eblocks((long long)v2 * 64), 256, 0, u->st>>>(u->e3, 64, n3, b, u->u3);
  CK(conv(u, n2, v2, u->u3, 64, u->e2, 32, u->wf[L_D2A], u->bias[L_D2A], 3, u->a4a, 32, nullptr, 0, true, false));
  CK(conv(u, n2, v2, u->a4a, 32, nullptr, 0, u->wf[L_D2B], u->bias[L_D2B], 3, u->g2, 32, nullptr, 0, true, false));
  k_up<<<eblocks((long long)v1 * 32), 256, 0, u->st>>>(u->g2, 32, n2, b, u->u2);
  CK(conv(u, n1, v1, u->u2, 32, u->e1, 16, u->wf[L_D1A], u->bias[L_D1A], 3, u->a5a, 16, nullptr, 0, true, false));
  CK(conv(u, n1, v1, u->a5a, 16, nullptr, 0, u->wf[L_D1B], u->bias[L_D1B], 3, u->g1, 16, nullptr, 0, true, false));
  CK(conv(u, n1, v1, u->g1, 16, nullptr, 0, u->wf[L_HEAD], u->bias[L_HEAD], 1, u->y, 8, nullptr, 0, false, true));
  return cudaGetLastError();
}

// backward through one block B(.; a->c) with input [in0, in1], first conv la,
// second lb, outputs post_a (first activation) and post_b; gout is the
// gradient at post_b.  Writes the input gradient to gin0 / gin1 (if given).
cudaError_t block_back(les_unet* u, int la, int lb, int ln, int nvox, const bf16* in0, int c0, const bf16* in1, int c1,
                       const bf16* post_a, const bf16* post_b, const bf16* gout, bf16* gin0, bf16* gin1, bf16* s1,
                       bf16* s2) {
  const int ca = pad8(kLayers[la].cout), cb = pad8(kLayers[lb].cout);
  cudaError_t e;
  k_act_bwd<<<eblocks((long long)nvox * cb), 256, 0, u->st>>>(post_b, gout, (long long)nvox * cb, s1);
  CK(wgrad(u, lb, ln, nvox, s1, cb, post_a, ca, nullptr, 0));
  CK(conv(u, ln, nvox, s1, cb, nullptr, 0, u->wb[lb], nullptr, 3, s2, ca, nullptr, 0, false, false));
  k_act_bwd<<<eblocks((long long)nvox * ca), 256, 0, u->st>>>(post_a, s2, (long long)nvox * ca, s1);
  CK(wgrad(u, la, ln, nvox, s1, ca, in0, c0, in1, c1));
  if (gin0) CK(conv(u, ln, nvox, s1, ca, nullptr, 0, u->wb[la], nullptr, 3, gin0, c0, gin1, c1, false, false));
  return cudaGetLastError();
}

// full backward from gy (in G0, [v1][16], channel 0 real); fills u->grad
cudaError_t backward(les_unet* u, int b) {
  const int n1 = u->n, n2 = n1 / 2, n3 = n2 / 2;
  const int v1 = b * n1 * n1 * n1, v2 = v1 / 8, v3 = v2 / 8;
  cudaError_t e;
  bf16 *gy = u->G0, *gA = u->G1, *gB = u->G2, *s1 = u->G3, *s2 = u->G4;
  // head (1x1, no activation): weight grad and gradient at g1
  CK(wgrad(u, L_HEAD, n1, v1, gy, 16, u->g1, 16, nullptr, 0));
  CK(conv(u, n1, v1, gy, 16, nullptr, 0, u->wb[L_HEAD], nullptr, 1, gA, 16, nullptr, 0, false, false));
  // D1: input [u2 (32), e1 (16)] -> grads g_u2 (gB, 32 ch) and g_e1 (gy reused, 16 ch)
  bf16* g_e1 = gy;
  CK(block_back(u, L_D1A, L_D1B, n1, v1, u->u2, 32, u->e1, 16, u->a5a, u->g1, gA, gB, g_e1, s1, s2));
  // up backward: g_g2 (v2 x 32) into gA
  k_up_bwd<<<eblocks((long long)v2 * 32), 256, 0, u->st>>>(gB, 32, n2, b, gA);
  // D2: input [u3 (64), e2 (32)] -> g_u3 (gB, v2 x 64), g_e2 (s2... keep in a dedicated slot)
  bf16* g_e2 = u->G4 + (size_t)v1 * 32;  // tail of the last scratch buffer
  CK(block_back(u, L_D2A, L_D2B, n2, v2, u->u3, 64, u->e2, 32, u->a4a, u->g2, gA, gB, g_e2, s1, s2));
  k_up_bwd<<<eblocks((long long)v3 * 64), 256, 0, u->st>>>(gB, 64, n3, b, gA);  // g_e3
  // L3: input p2 (32) -> g_p2 (gB, v3 x 32)
  CK(block_back(u, L_E3A, L_E3B, n3, v3, u->p2, 32, nullptr, 0, u->a3a, u->e3, gA, gB, nullptr, s1, s2));
  k_pool_bwd<<<eblocks((long long)v2 * 32), 256, 0, u->st>>>(gB, 32, n2, b, g_e2, 1);
  // L2: input p1 (16) -> g_p1 (gB, v2 x 16)
  CK(block_back(u, L_E2A, L_E2B, n2, v2, u->p1, 16, nullptr, 0, u->a2a, u->e2, g_e2, gB, nullptr, s1, s2));
  k_pool_bwd<<<eblocks((long long)v1 * 16), 256, 0, u->st>>>(gB, 16, n1, b, g_e1, 1);
  // L1: input x0 (16, channel 0 real); its gradient is not needed
  CK(block_back(u, L_E1A, L_E1B, n1, v1, u->x0, 16, nullptr, 0, u->a1a, u->e1, g_e1, nullptr, nullptr, s1, s2));
  return cudaGetLastError();
#undef CK
}

template <typename T>
cudaError_t pack_inputs(les_unet* u, const T* b, const T* psi, int batch) {
  const long long n3 = (long long)u->n * u->n * u->n;
  const int nblk = 64;
  k_sumsq<T><<<dim3(nblk, batch), 256, 0, u->st>>>(b, n3, u->dpart);
  k_scale<<<1, 64, 0, u->st>>>(u->dpart, nblk, n3, batch, u->scale);
  k_pack<T><<<eblocks(batch * n3), 256, 0, u->st>>>(b, psi, n3, batch, u->scale, u->out_scale, u->x0,
                                                     psi ? u->tgt : nullptr);
  return cudaGetLastError();
}

template <typename T>
int run_forward(les_unet* u, const T* b, int batch, T* psi0) {
  cudaError_t e;
  if ((e = pack_inputs<T>(u, b, (const T*)nullptr, batch)) != cudaSuccess) return unet_fail(u, e, "pack");
  if ((e = forward(u, batch)) != cudaSuccess) return unet_fail(u, e, "forward");
  const long long n3 = (long long)u->n * u->n * u->n;
  k_ymean<<<batch, 256, 0, u->st>>>(u->y, n3, u->ymean);
  k_unpack<T><<<eblocks(batch * n3), 256, 0, u->st>>>(u->y, n3, batch, u->scale, u->out_scale, u->ymean, psi0);
  e = cudaGetLastError();
  return e == cudaSuccess ? LES_OK : unet_fail(u, e, "unpack");
}

template <typename T>
int run_loss_grad(les_unet* u, const T* b, const T* psi, int batch, double* loss) {
  cudaError_t e;
  if ((e = pack_inputs<T>(u, b, psi, batch)) != cudaSuccess) return unet_fail(u, e, "pack");
  if ((e = forward(u, batch)) != cudaSuccess) return unet_fail(u, e, "forward");
  const long long total = (long long)batch * u->n * u->n * u->n;
  const int nb = (int)std::min<long long>((total + 255) / 256, 4096);
  if (u->loss_kind == 1) k_loss_energy<<<nb, 256, 0, u->st>>>(u->y, u->tgt, u->n, total, u->G0, u->dpart);
  else k_loss<<<nb, 256, 0, u->st>>>(u->y, u->tgt, total, u->G0, u->dpart);
  k_sum_part<<<1, 256, 0, u->st>>>(u->dpart, nb, u->loss);
  if ((e = backward(u, batch)) != cudaSuccess) return unet_fail(u, e, "backward");
  if (loss) {
    double h = 0;
    if ((e = cudaMemcpyAsync(&h, u->loss, 8, cudaMemcpyDeviceToHost, u->st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(u->st)) != cudaSuccess)
      return unet_fail(u, e, "loss readback");
    *loss = h / (double)total;
  }
  return LES_OK;
}

int check_n(int n) { return n >= 8 && n % 4 == 0 && n <= 512; }

}  // namespace

namespace les {
// used by the solver handle for LES_WARM_LEARNED
int unet_predict(les_unet* u, int precision, const void* b, void* psi0, cudaStream_t st, std::string* err) {
  u->st = st;
  const int rc = precision == 64 ? run_forward<double>(u, (const double*)b, 1, (double*)psi0)
                                 : run_forward<float>(u, (const float*)b, 1, (float*)psi0);
  if (rc != LES_OK && err) *err = u->err;
  return rc;
}
int unet_grid(const les_unet* u) { return u ? u->n : 0; }
}  // namespace les

extern "C" {

int64_t les_unet_param_count(void) {
  int64_t np = 0;
  for (int l = 0; l < kNL; ++l)
    np += (int64_t)kLayers[l].cout * kLayers[l].cin * kLayers[l].k * kLayers[l].k * kLayers[l].k + kLayers[l].cout;
  return np;
}

int les_unet_workspace_bytes(int32_t n, int32_t batch, size_t* bytes) {
  if (!bytes || !check_n(n) || batch < 1 || batch > 4096) return LES_ERR_INVALID_ARG;
  les_unet tmp;
  tmp.n = n;
  tmp.batch = batch;
  *bytes = layout(&tmp, nullptr, true);
  return LES_OK;
}

int les_unet_create(int32_t n, int32_t batch, void* workspace, size_t bytes, void* stream, les_unet** out) {
  if (!out) return LES_ERR_INVALID_ARG;
  *out = nullptr;
  size_t need = 0;
  if (les_unet_workspace_bytes(n, batch, &need) != LES_OK || !workspace || bytes < need ||
      ((uintptr_t)workspace % 256) != 0)
    return LES_ERR_INVALID_ARG;
  les_unet* u = new (std::nothrow) les_unet();
  if (!u) return LES_ERR_INVALID_ARG;
  u->n = n;
  u->batch = batch;
  u->st = (cudaStream_t)stream;
  u->ws = (char*)workspace;
  u->ws_bytes = bytes;
  layout(u, u->ws, false);
  cudaError_t e = cudaMemsetAsync(u->ws, 0, need, u->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->st);
  if (e != cudaSuccess) {
    delete u;
    return LES_ERR_CUDA;
  }
  *out = u;
  return LES_OK;
}

void les_unet_destroy(les_unet* u) { delete u; }

int les_unet_set_stream(les_unet* u, void* stream) {
  if (!u) return LES_ERR_INVALID_ARG;
  u->st = (cudaStream_t)stream;
  return LES_OK;
}

int les_unet_set_weights(les_unet* u, const float* w, int32_t on_device) {
  if (!u || !w) return LES_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(u->master, w, u->nparams * 4,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, u->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->m1, 0, u->nparams * 4, u->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(u->m2, 0, u->nparams * 4, u->st);
  if (e == cudaSuccess) e = refresh_weights(u);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(u->st);
  u->step = 0;
  return e == cudaSuccess ? LES_OK : unet_fail(u, e, "set_weights");
}

int les_unet_get_weights(les_unet* u, float* w, int32_t on_device) {
  if (!u || !w) return LES_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpyAsync(w, u->master, u->nparams * 4,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, u->st);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(u->st);
  return e == cudaSuccess ? LES_OK : unet_fail(u, e, "get_weights");
}

int les_unet_forward(les_unet* u, int32_t precision, const void* d_b, int32_t batch, void* d_psi0) {
  if (!u || !d_b || !d_psi0 || batch < 1 || batch > u->batch || (precision != 32 && precision != 64))
    return LES_ERR_INVALID_ARG;
  return precision == 64 ? run_forward<double>(u, (const double*)d_b, batch, (double*)d_psi0)
                         : run_forward<float>(u, (const float*)d_b, batch, (float*)d_psi0);
}

int les_unet_loss_grad(les_unet* u, int32_t precision, const void* d_b, const void* d_psi, int32_t batch,
                       double* loss, float* d_grad) {
  if (!u || !d_b || !d_psi || batch < 1 || batch > u->batch || (precision != 32 && precision != 64))
    return LES_ERR_INVALID_ARG;
  int rc = precision == 64 ? run_loss_grad<double>(u, (const double*)d_b, (const double*)d_psi, batch, loss)
                           : run_loss_grad<float>(u, (const float*)d_b, (const float*)d_psi, batch, loss);
  if (rc == LES_OK && d_grad) {
    cudaError_t e = cudaMemcpyAsync(d_grad, u->grad, u->nparams * 4, cudaMemcpyDeviceToDevice, u->st);
    if (e != cudaSuccess) return unet_fail(u, e, "grad copy");
  }
  return rc;
}

int les_unet_train_step(les_unet* u, int32_t precision, const void* d_b, const void* d_psi, int32_t batch, float lr,
                        double* loss) {
  int rc = les_unet_loss_grad(u, precision, d_b, d_psi, batch, loss, nullptr);
  if (rc != LES_OK) return rc;
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
  {
    ProfScope ps(u->prof, KI_UNET_ADAM, u->st);
    k_adam<<<eblocks((long long)u->nparams), 256, 0, u->st>>>(u->master, u->grad, u->m1, u->m2,
                                                              (long long)u->nparams, lr, b1, b2, 1e-8f, c1, c2);
  }
  cudaError_t e = refresh_weights(u);
  return e == cudaSuccess ? LES_OK : unet_fail(u, e, "adam");
}

int les_unet_set_loss(les_unet* u, int32_t kind) {
  if (!u || (kind != LES_UNET_LOSS_MSE && kind != LES_UNET_LOSS_ENERGY)) return LES_ERR_INVALID_ARG;
  u->loss_kind = kind;
  return LES_OK;
}

int les_unet_set_output_scale(les_unet* u, double scale) {
  if (!u || !(scale > 0) || !std::isfinite(scale)) return LES_ERR_INVALID_ARG;
  u->out_scale = scale;
  return LES_OK;
}

double les_unet_get_output_scale(const les_unet* u) { return u ? u->out_scale : 0.0; }

const char* les_unet_last_error(const les_unet* u) { return u ? u->err.c_str() : "no model"; }

}  // extern "C"
