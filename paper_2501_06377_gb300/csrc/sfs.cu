// sfs.cu -- the learned one-day surrogate (include/sfs.h): the network's
// training forward and backward passes, AdamW, and the C-ABI.
//
// Every contraction of the training pass is a BF16 x BF16 -> FP32 product on
// the tcgen05 tensor cores (sfs_gemm.cu): batched by strides (a zero stride
// shares an operand), either operand K-major or MN-major, split-K for the
// weight gradients (K = batch x tokens).  Activations that only ever feed a
// product (the embedding E, the spectral outputs Yh and dHh, the GELU
// outputs A, the decoder gradient dD and the pre-activation gradient dZ)
// are stored in BF16, which is the precision the product reads them in, so
// they cost half the bytes and reach shared memory by TMA; the residual
// stream and its gradient stay FP32.  The fixed rotation layer is an FFT per
// map row (rot_fft_kernel), not a GEMM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sfs.h"
#include "sfs_fused.cuh"
#include "sfs_gemm.cuh"
#include <nvtx3/nvToolsExt.h>

namespace sft {
void set_global_error(const std::string& msg);
}

namespace {

constexpr int H = 256, W = 512, PATCH = 4, HT = H / PATCH, WT = W / PATCH, KE = 48;
constexpr int NTOK = HT * WT;           // tokens per map
constexpr float SCALE = 100.0f;         // map normalisation (G)
constexpr int kRedBlocks = 64;          // blocks per map of the per-map reductions
constexpr double PI = 3.14159265358979323846;

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint2 pack4(float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

// ---------------------------------------------------------------------------
// GEMM (sfs_gemm.cu: tcgen05 tensor cores, TMEM accumulators, TMA for the
// BF16 operands); the split-K partial products are folded here
// ---------------------------------------------------------------------------
// out[i] = beta * out[i] + sum_q part[q * n + i], q < ns: one warp per
// output, lane l adding q = l, l + 32, ... in order and a fixed shuffle tree
// combining the lanes (deterministic, independent of the launch shape).
__global__ void fold_parts_kernel(const float* __restrict__ part, int ns, long long n, float beta,
                                  float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    float s = 0.f;
    for (int q = lane; q < ns; q += 32) s += part[(long long)q * n + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = (beta != 0.f ? beta * out[i] : 0.f) + s;
  }
}

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&v)[4]) {
  const uint2 t = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&t.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&t.y);
  v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
}

// Column sums of X[rows][ncols] (the bias gradients): block b adds its
// contiguous row range into part[b][ncols] in a fixed order (four columns
// per thread, ncols / 4 threads per row, the row offsets folded in order
// through shared memory).  ncols divides 1024 and is a multiple of 4.
template <typename T>
__global__ void __launch_bounds__(256) colsum_part_kernel(const T* __restrict__ X, long long rows, int ncols,
                                                         float* __restrict__ part) {
  __shared__ float sh[1024];
  const int tpr = ncols / 4, c4 = (threadIdx.x % tpr) * 4, rl = threadIdx.x / tpr, rstep = blockDim.x / tpr;
  const long long per = (rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = (long long)blockIdx.x * per, r1 = min(rows, r0 + per);
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (long long r = r0 + rl; r < r1; r += rstep) {
    float v[4];
    load4(X + r * ncols + c4, v);
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] += v[e];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) sh[rl * ncols + c4 + e] = acc[e];
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < rstep; ++q) s += sh[q * ncols + c];
    part[(long long)blockIdx.x * ncols + c] = s;
  }
}

// ---------------------------------------------------------------------------
// elementwise kernels of the network
// ---------------------------------------------------------------------------
// alpha[b*H + j]: the day's rotation angle of row j (FP64), from
// Omega(lat) = o0 + o2 sin^2 lat + o4 sin^4 lat - 360/27.2753 deg/day.
__global__ void rot_angle_kernel(const float* __restrict__ p, int rows, double* __restrict__ alpha) {
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < rows; row += gridDim.x * blockDim.x) {
    const int b = row / H, j = row % H;
    const double c = cos(j * (PI / (H - 1)));
    const double s2 = c * c;
    const double om = p[5 * b + 0] + p[5 * b + 1] * s2 + p[5 * b + 2] * s2 * s2 - 360.0 / 27.2753;
    alpha[row] = om * (PI / 180.0);
  }
}

// Layer R by FFT: the 512-point DFT X of the real row, Y_k = X_k
// exp(-i k alpha_row) on modes 0..256, the Hermitian extension Y_{512-k} =
// conj(Y_k) (the Nyquist mode keeps its real part only, as the truncated
// synthesis G does), and the inverse transform scaled by 1/512, taken as
// Re(DFT(conj Y)) / 512.  The same map as r = phase(x F^T) G^T, in FP32 with
// O(log n) rounding.
//
// Each DFT is three radix-8 passes of the Stockham autosort formulation
// (Govindaraju et al., SC 2008): with Ns = 1, 8, 64, butterfly j (0..63)
// reads v_q = a[j + 64 q], multiplies v_q by exp(-2 pi i q (j mod Ns) /
// (8 Ns)), takes the 8-point DFT and writes it to b[(j / Ns) 8 Ns + (j mod Ns)
// + q Ns]; after the third pass butterfly j holds X_{j + 64 q} in order.  A
// block of 256 threads transforms 4 rows (64 threads each); the passes
// exchange through shared memory.  tw[j] = exp(-2 pi i j / 512), j < 256.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// in-place 8-point DFT (exponent sign -1): two radix-2 layers and radix-4
// DFTs of the even and odd outputs
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  constexpr float c = 0.70710678118654752f;
  float2 a[4], b[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = make_float2(v[k].x + v[k + 4].x, v[k].y + v[k + 4].y);
    b[k] = make_float2(v[k].x - v[k + 4].x, v[k].y - v[k + 4].y);
  }
  // b_k *= exp(-2 pi i k / 8)
  b[1] = make_float2(c * (b[1].x + b[1].y), c * (b[1].y - b[1].x));
  b[2] = make_float2(b[2].y, -b[2].x);
  b[3] = make_float2(c * (b[3].y - b[3].x), -c * (b[3].x + b[3].y));
  float2* io[2] = {a, b};
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // 4-point DFTs: outputs 2m + h
    const float2* x = io[h];
    const float2 s02 = make_float2(x[0].x + x[2].x, x[0].y + x[2].y), d02 = make_float2(x[0].x - x[2].x, x[0].y - x[2].y);
    const float2 s13 = make_float2(x[1].x + x[3].x, x[1].y + x[3].y), d13 = make_float2(x[1].x - x[3].x, x[1].y - x[3].y);
    v[h] = make_float2(s02.x + s13.x, s02.y + s13.y);
    v[4 + h] = make_float2(s02.x - s13.x, s02.y - s13.y);
    v[2 + h] = make_float2(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
    v[6 + h] = make_float2(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
  }
}

// One Stockham radix-8 pass of butterfly j on shared rows: a -> v -> b.
template <int NS>
__device__ __forceinline__ void stockham_pass(const float2* a, float2* b, const float2* tws, int j, float2 (&v)[8],
                                              bool write) {
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = a[j + 64 * q];
  if (NS > 1) {
    const int e0 = (j % NS) * (512 / (8 * NS));  // exponent step (units of 2 pi / 512)
#pragma unroll
    for (int q = 1; q < 8; ++q) {
      const int e = q * e0;  // < 512
      const float2 w = e < 256 ? tws[e] : make_float2(-tws[e - 256].x, -tws[e - 256].y);
      v[q] = cmul(v[q], w);
    }
  }
  dft8(v);
  if (write) {
    const int base = (j / NS) * 8 * NS + (j % NS);
#pragma unroll
    for (int q = 0; q < 8; ++q) b[base + NS * q] = v[q];
  }
}

__global__ void __launch_bounds__(256) rot_fft_kernel(const float* __restrict__ x, const double* __restrict__ alpha,
                                                      const float2* __restrict__ tw, int rows, float* __restrict__ r) {
  static_assert(W == 512, "rot_fft_kernel is written for 512-point rows");
  __shared__ float2 tws[256];
  __shared__ float2 s0[4][W], s1[4][W];
  const int t = threadIdx.x, q4 = t >> 6, j = t & 63;
  const int row = blockIdx.x * 4 + q4;
  const bool live = row < rows;
  tws[t] = tw[t];
  float2 v[8];
  // pass 1 (Ns = 1) straight from the real row in global memory
  const float* xr = x + (long long)(live ? row : 0) * W;
#pragma unroll
  for (int q = 0; q < 8; ++q) v[q] = make_float2(live ? xr[j + 64 * q] : 0.f, 0.f);
  dft8(v);
#pragma unroll
  for (int q = 0; q < 8; ++q) s0[q4][8 * j + q] = v[q];
  __syncthreads();
  stockham_pass<8>(s0[q4], s1[q4], tws, j, v, true);
  __syncthreads();
  stockham_pass<64>(s1[q4], nullptr, tws, j, v, false);  // v[q] = X_{j + 64 q}
  // phase on modes k = j + 64 q <= 256, Hermitian extension into s0
  const double a = live ? alpha[row] : 0.0;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int k = j + 64 * q;
    if (k > W / 2) break;
    const double ang = k * a;
    const double red = ang - (2.0 * PI) * rint(ang * (1.0 / (2.0 * PI)));  // in [-pi, pi]
    float sn, cs;
    sincosf((float)red, &sn, &cs);
    const float2 X = v[q];
    const float2 Y = make_float2(X.x * cs + X.y * sn, X.y * cs - X.x * sn);
    if (k == W / 2) {
      s0[q4][k] = make_float2(Y.x, 0.f);
    } else {
      s0[q4][k] = Y;
      if (k > 0) s0[q4][W - k] = make_float2(Y.x, -Y.y);
    }
  }
  __syncthreads();
  // inverse: the forward DFT of conj(Y), real part / 512
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float2 y = s0[q4][j + 64 * q];
    v[q] = make_float2(y.x, -y.y);
  }
  dft8(v);
#pragma unroll
  for (int q = 0; q < 8; ++q) s1[q4][8 * j + q] = v[q];
  __syncthreads();
  stockham_pass<8>(s1[q4], s0[q4], tws, j, v, true);
  __syncthreads();
  stockham_pass<64>(s0[q4], nullptr, tws, j, v, false);  // v[q] = Z_{j + 64 q}
  if (live) {
    float* rr = r + (long long)row * W;
    constexpr float inv = 1.0f / W;
#pragma unroll
    for (int q = 0; q < 8; ++q) rr[j + 64 * q] = v[q].x * inv;
  }
}

// E[token][48]: 4x4 patches of x/s and r/s, normalised parameters, cos/sin of
// the patch-row colatitude, zeros.  One thread per token.
__global__ void embed_kernel(const float* __restrict__ x, const float* __restrict__ r,
                             const float* __restrict__ p, int nb, bf16* __restrict__ E) {
  const long long n = (long long)nb * NTOK;
  const float ref[5] = {13.38f, -2.30f, -1.62f, 15.0f, 500.0f};
  const float spr[5] = {1.338f, 0.230f, 0.162f, 5.0f, 250.0f};
  for (long long tok = blockIdx.x * (long long)blockDim.x + threadIdx.x; tok < n;
       tok += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(tok / NTOK), t = (int)(tok % NTOK);
    const int i = t / WT, l = t % WT;
    uint2* out = reinterpret_cast<uint2*>(E + tok * KE);
    const float inv = 1.0f / SCALE;
#pragma unroll
    for (int pr = 0; pr < PATCH; ++pr) {
      const long long off = ((long long)b * H + i * PATCH + pr) * W + l * PATCH;
      float4 vx = *reinterpret_cast<const float4*>(x + off);
      float4 vr = *reinterpret_cast<const float4*>(r + off);
      vx.x *= inv; vx.y *= inv; vx.z *= inv; vx.w *= inv;
      vr.x *= inv; vr.y *= inv; vr.z *= inv; vr.w *= inv;
      out[pr] = pack4(vx.x, vx.y, vx.z, vx.w);
      out[4 + pr] = pack4(vr.x, vr.y, vr.z, vr.w);
    }
    const float q0 = (p[5 * b + 0] - ref[0]) / spr[0], q1 = (p[5 * b + 1] - ref[1]) / spr[1];
    const float q2 = (p[5 * b + 2] - ref[2]) / spr[2], q3 = (p[5 * b + 3] - ref[3]) / spr[3];
    const float q4 = (p[5 * b + 4] - ref[4]) / spr[4];
    const double th = (i + 0.5) * PATCH * (PI / (H - 1));
    out[8] = pack4(q0, q1, q2, q3);
    out[9] = pack4(q4, (float)cos(th), (float)sin(th), 0.f);
    out[10] = make_uint2(0u, 0u);
    out[11] = make_uint2(0u, 0u);
  }
}

// Yh = w (.) Hh per (latent row i, mode k, channel c); layout [(b*HT+i)][2M][C].
__global__ void spectral_fwd_kernel(const float* __restrict__ Hh, const float* __restrict__ w, int nb, int M,
                                    int C, bf16* __restrict__ Yh) {
  const long long n = (long long)nb * HT * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int k = (int)((e / C) % M);
    const long long bi = e / ((long long)C * M);
    const int i = (int)(bi % HT);
    const float* hp = Hh + bi * 2 * M * C;
    bf16* yp = Yh + bi * 2 * M * C;
    const float hr = hp[(long long)k * C + c], hi = hp[(long long)(M + k) * C + c];
    const float wr = w[(((long long)i * M + k) * C + c) * 2], wi = w[(((long long)i * M + k) * C + c) * 2 + 1];
    yp[(long long)k * C + c] = __float2bfloat16_rn(wr * hr - wi * hi);
    yp[(long long)(M + k) * C + c] = __float2bfloat16_rn(wr * hi + wi * hr);
  }
}

// dHh = conj-transpose action of w on dYh.
__global__ void spectral_bwd_x_kernel(const float* __restrict__ dYh, const float* __restrict__ w, int nb, int M,
                                      int C, bf16* __restrict__ dHh) {
  const long long n = (long long)nb * HT * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int k = (int)((e / C) % M);
    const long long bi = e / ((long long)C * M);
    const int i = (int)(bi % HT);
    const float* dp = dYh + bi * 2 * M * C;
    bf16* op = dHh + bi * 2 * M * C;
    const float dr = dp[(long long)k * C + c], di = dp[(long long)(M + k) * C + c];
    const float wr = w[(((long long)i * M + k) * C + c) * 2], wi = w[(((long long)i * M + k) * C + c) * 2 + 1];
    op[(long long)k * C + c] = __float2bfloat16_rn(wr * dr + wi * di);
    op[(long long)(M + k) * C + c] = __float2bfloat16_rn(-wi * dr + wr * di);
  }
}

// gw[i][k][c][2] = sum over the batch (fixed order).
__global__ void spectral_bwd_w_kernel(const float* __restrict__ dYh, const float* __restrict__ Hh, int nb, int M,
                                      int C, float* __restrict__ gw) {
  const long long n = (long long)HT * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int k = (int)((e / C) % M);
    const int i = (int)(e / ((long long)C * M));
    float sr = 0.f, si = 0.f;
    for (int b = 0; b < nb; ++b) {
      const long long base = ((long long)b * HT + i) * 2 * M * C;
      const float hr = Hh[base + (long long)k * C + c], hi = Hh[base + (long long)(M + k) * C + c];
      const float dr = dYh[base + (long long)k * C + c], di = dYh[base + (long long)(M + k) * C + c];
      sr += dr * hr + di * hi;
      si += -dr * hi + di * hr;
    }
    gw[e * 2] = sr;
    gw[e * 2 + 1] = si;
  }
}

__device__ __forceinline__ float gelu_f(float z) {
  const float c = 0.7978845608028654f;
  return 0.5f * z * (1.f + tanhf(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_g(float z) {
  const float c = 0.7978845608028654f;
  const float t = tanhf(c * (z + 0.044715f * z * z * z));
  return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * c * (1.f + 3.f * 0.044715f * z * z);
}

__global__ void gelu_fwd_kernel(const float* __restrict__ z, long long n, bf16* __restrict__ a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    a[e] = __float2bfloat16_rn(gelu_f(z[e]));
}

__global__ void gelu_bwd_kernel(const float* __restrict__ da, const float* __restrict__ z, long long n,
                                bf16* __restrict__ dz) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dz[e] = __float2bfloat16_rn(da[e] * gelu_g(z[e]));
}

// delta map from the decoder's patches: out[b][row][col] = d[token][4 pr + pc]
__global__ void unpatch_kernel(const float* __restrict__ d, int nb, float* __restrict__ out) {
  const long long n = (long long)nb * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / (H * W)), rem = (int)(e % (H * W));
    const int row = rem / W, col = rem % W;
    const long long tok = (long long)b * NTOK + (row / PATCH) * WT + col / PATCH;
    out[e] = d[tok * 16 + (row % PATCH) * PATCH + col % PATCH];
  }
}

// x_next = r + s (delta - <delta>_A) in place over delta; msum[2b] = sum A delta.
__global__ void center_kernel(float* __restrict__ xn, const float* __restrict__ r,
                              const double* __restrict__ msum, double area_total, int nb) {
  // block row blockIdx.y is map b: its mean (an FP64 division) is formed once per thread
  const int b = blockIdx.y;
  const float mean = (float)(msum[2 * b] / area_total);
  float* xm = xn + (long long)b * H * W;
  const float* rm = r + (long long)b * H * W;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * W; e += gridDim.x * blockDim.x)
    xm[e] = rm[e] + SCALE * (xm[e] - mean);
}

// Per map m, block partials of sum (x - y)^2, sum y^2, sum (x - y) (three per block).
__global__ void loss_sums_kernel(const float* __restrict__ x, const float* __restrict__ y,
                                 double* __restrict__ out) {
  __shared__ double s0[256], s1[256], s2[256];
  const int m = blockIdx.y;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)H * W;
       e += (long long)gridDim.x * blockDim.x) {
    const double d = double(x[(long long)m * H * W + e]) - double(y[(long long)m * H * W + e]);
    const double yv = y[(long long)m * H * W + e];
    a0 += d * d;
    a1 += yv * yv;
    a2 += d;
  }
  s0[threadIdx.x] = a0;
  s1[threadIdx.x] = a1;
  s2[threadIdx.x] = a2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {  // this block's partials; fold_map_sums adds them in a fixed order
    double* q = out + ((long long)m * gridDim.x + blockIdx.x) * 3;
    q[0] = s0[0];
    q[1] = s1[0];
    q[2] = s2[0];
  }
}

__global__ void sumsq_kernel(const float* __restrict__ a, const float* __restrict__ b, int nb,
                             double* __restrict__ out) {
  // block partials of sum (a-b)^2 and sum b^2 for map m (b may be null: then a^2 only)
  __shared__ double s0[256], s1[256];
  const int m = blockIdx.y;
  double x0 = 0.0, x1 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)H * W;
       e += (long long)gridDim.x * blockDim.x) {
    const float av = a[(long long)m * H * W + e];
    const float bv = b ? b[(long long)m * H * W + e] : 0.f;
    x0 += double(av - bv) * double(av - bv);
    x1 += double(bv) * double(bv);
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* q = out + ((long long)m * gridDim.x + blockIdx.x) * 2;
    q[0] = s0[0];
    q[1] = s1[0];
  }
  (void)nb;
}

// dd[token][16]: the loss gradient g = 2 (x_next - y) / (||y||^2 n) through
// the centring: s (g - A_row sum(g) / sum(A)).  Block row blockIdx.y is map
// b, whose two FP64 constants each thread forms once.
__global__ void loss_grad_kernel(const float* __restrict__ xn, const float* __restrict__ y,
                                 const double* __restrict__ sums, const double* __restrict__ area,
                                 double area_total, int nb, bf16* __restrict__ dd) {
  const int b = blockIdx.y;
  const double k = 2.0 / (sums[3 * b + 1] * nb);
  const double gs = k * sums[3 * b + 2] / area_total;
  const float* xm = xn + (long long)b * H * W;
  const float* ym = y + (long long)b * H * W;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H * W; e += gridDim.x * blockDim.x) {
    const int row = e / W, col = e % W;
    const long long tok = (long long)b * NTOK + (row / PATCH) * WT + col / PATCH;
    const double g = k * (double(xm[e]) - double(ym[e]));
    dd[tok * 16 + (row % PATCH) * PATCH + col % PATCH] = __float2bfloat16_rn((float)(SCALE * (g - area[row] * gs)));
  }
}

// Per map m: block partials of sum A B and sum A |B| (FP64) with the
// 256 x 512 grid's area weights (sin th_j dth dph; the pole rows share the
// cap area 2 pi (1 - cos(dth/2)) over their nphi entries).
__global__ void flux_kernel(const float* __restrict__ a, const double* __restrict__ area,
                            double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  const int m = blockIdx.y;
  double x0 = 0.0, x1 = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)H * W;
       e += (long long)gridDim.x * blockDim.x) {
    const double v = a[(long long)m * H * W + e];
    const double w = area[e / W];
    x0 += w * v;
    x1 += w * fabs(v);
  }
  s0[threadIdx.x] = x0;
  s1[threadIdx.x] = x1;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s0[threadIdx.x] += s0[threadIdx.x + o];
      s1[threadIdx.x] += s1[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double* q = out + ((long long)m * gridDim.x + blockIdx.x) * 2;
    q[0] = s0[0];
    q[1] = s1[0];
  }
}

// out[m][f] = sum over the nblk block partials of map m, in block order
// (deterministic, unlike atomics).
__global__ void fold_map_sums(const double* __restrict__ part, int nblk, int k, double* __restrict__ out) {
  const int m = blockIdx.x, f = threadIdx.x;
  if (f >= k) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[((long long)m * nblk + b) * k + f];
  out[(long long)m * k + f] = acc;
}

__global__ void adamw_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                             float* __restrict__ v, long long n, float lr, float wd, float bc1, float bc2) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = 0.9f * m[e] + 0.1f * gi;
    const float vi = 0.999f * v[e] + 0.001f * gi * gi;
    m[e] = mi;
    v[e] = vi;
    const float mh = mi / bc1, vh = vi / bc2;
    p[e] -= lr * (mh / (sqrtf(vh) + 1e-8f) + wd * p[e]);
  }
}


int grid_for(long long n) { return (int)std::min<long long>((n + 255) / 256, 152LL * 16); }

}  // namespace

struct sfs_net {
  int C = 0, M = 0, L = 0, maxb = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // parameters (flat): offsets
  long long oWe, obe, oWd, obd;
  std::vector<long long> ow, oW1, ob1, oW2, ob2;
  long long np = 0;
  float *P = nullptr, *G = nullptr, *Mo = nullptr, *Vo = nullptr;
  int t = 0;
  // fixed matrices
  float *Fm = nullptr, *Gm = nullptr;
  float2* tw = nullptr;  // FFT twiddles exp(-2 pi i j / W), j < W/2
  // activations
  // (BF16: the activations that only feed products)
  float *R = nullptr, *D = nullptr, *XN = nullptr;
  bf16* E = nullptr;
  std::vector<float*> Hs, Hh, U, Z;
  std::vector<bf16*> A;
  bf16* Yh = nullptr;
  // gradients of activations
  float *dH = nullptr, *dU = nullptr, *dA = nullptr, *dYh = nullptr;
  bf16 *dD = nullptr, *dZ = nullptr, *dHh = nullptr;
  int* gerr = nullptr;   // device: nonzero once a GEMM wait ran out of time
  int* hgerr = nullptr;  // pinned host copy
  float* part = nullptr;
  long long part_elems = 0;
  double* sums = nullptr;
  double* hbig = nullptr;  // pinned staging of the chunked reductions
  long long hbig_n = 0;
  double* area = nullptr;   // per-row area weight of one entry
  double* alpha = nullptr;  // per (map, row) rotation angle
  double area_total = 0.0;  // sum of the weights over the whole map
  double* msum = nullptr;   // per map: sum A delta (output centring)
  double* mpart = nullptr;  // per map and reduction block: partial sums (kRedBlocks x 3)
  double* lsum = nullptr;   // per map: loss sums
  double* hlsum = nullptr;
  int64_t gemms = 0, kernels = 0;
  double flops = 0.0;
  std::vector<void*> allocs;
  // fused inference forward (C = 64, M = 48, L <= 4): BF16 weight image,
  // rebuilt when the parameters change (pver counts the changes)
  bool fused = false;
  unsigned char* img = nullptr;
  long long pver = 0, img_pver = -1;
  int n_sm = 0;
  int sm_budget = 0;  // > 0: the fused forward's persistent blocks (SMs) are capped at this
  sfs_fused::ParamOffsets po{};
};

namespace {

sft_status fail(const std::string& m, sft_status c = SFT_ERR_CUDA) {
  sft::set_global_error(m);
  return c;
}

#define SFS_CUDA(call)                                                                             \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return fail(std::string(#call) + ": " + cudaGetErrorString(e_),                              \
                  e_ == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA);                   \
  } while (0)

template <typename T>
sft_status dalloc(sfs_handle h, T** p, long long n) {
  SFS_CUDA(cudaMalloc(p, std::max<long long>(n, 1) * sizeof(T)));
  h->allocs.push_back(*p);
  return SFT_OK;
}

// Operands of a product: element (mn, k) at p[mn*ld + k] (KMAJ) or at
// p[k*ld + mn] (MNMAJ), batch stride s (0: shared by every batch).
constexpr int KMAJ = 0, MNMAJ = 1;
sfs_gemm::Operand opnd(const float* p, long long ld, long long s, int major) {
  return sfs_gemm::Operand{p, sfs_gemm::F32, major, ld, s};
}
sfs_gemm::Operand opnd(const bf16* p, long long ld, long long s, int major) {
  return sfs_gemm::Operand{p, sfs_gemm::BF16, major, ld, s};
}

// C = alpha A B + beta C + bias (A: M x K, B: K x N), batched by strides.
sft_status gemm(sfs_handle h, int M, int N, int K, const sfs_gemm::Operand& a, const sfs_gemm::Operand& b, float* C,
                long long ldc, long long sC, float alpha, float beta, const float* bias, int batch) {
  sfs_gemm::Problem pr{M, N, K, a, b, C, ldc, sC, alpha, beta, bias, 0, batch};
  SFS_CUDA(sfs_gemm::launch(pr, h->gerr, h->stream));
  h->gemms += 1;
  h->kernels += 1;
  h->flops += 2.0 * M * N * (double)K * batch;
  return SFT_OK;
}

// Weight gradient C[M][N] (ldc = N) = A B with a long K: split-K into
// partial products, then a fixed-order reduction.
sft_status gemm_wgrad(sfs_handle h, int M, int N, int K, const sfs_gemm::Operand& a, const sfs_gemm::Operand& b,
                      float* C) {
  const int kchunk = 1024;
  const int ns = (K + kchunk - 1) / kchunk;
  if ((long long)ns * M * N > h->part_elems) return fail("split-K scratch too small", SFT_ERR_ARG);
  sfs_gemm::Problem pr{M, N, K, a, b, h->part, N, (long long)M * N, 1.f, 0.f, nullptr, kchunk, ns};
  SFS_CUDA(sfs_gemm::launch(pr, h->gerr, h->stream));
  fold_parts_kernel<<<grid_for((long long)M * N * 32), 256, 0, h->stream>>>(h->part, ns, (long long)M * N, 0.f, C);
  SFS_CUDA(cudaGetLastError());
  h->gemms += 1;
  h->kernels += 2;
  h->flops += 2.0 * M * N * (double)K;
  return SFT_OK;
}

// Bias gradient out[c] = sum over the ntok rows of X[row][c] (fixed order).
template <typename T>
sft_status bias_grad(sfs_handle h, const T* X, long long rows, int ncols, float* out) {
  const int nblk = 256;
  if ((long long)nblk * ncols > h->part_elems) return fail("column-sum scratch too small", SFT_ERR_ARG);
  colsum_part_kernel<T><<<nblk, 256, 0, h->stream>>>(X, rows, ncols, h->part);
  fold_parts_kernel<<<grid_for((long long)ncols * 32), 256, 0, h->stream>>>(h->part, nblk, ncols, 0.f, out);
  SFS_CUDA(cudaGetLastError());
  h->kernels += 2;
  return SFT_OK;
}

// A GEMM wait that ran out of time leaves a code in h->gerr; read it with the
// step's other results (after a stream synchronisation).
sft_status check_gemm_error(sfs_handle h) {
  if (*h->hgerr != 0) return fail("tensor-core GEMM: a wait inside the kernel ran out of time", SFT_ERR_CUDA);
  return SFT_OK;
}

// dft matrices (host FP64 -> device FP32): F [2m][n], G [n][2m]
void dft_host(int n, int m, std::vector<float>& F, std::vector<float>& G) {
  F.assign((size_t)2 * m * n, 0.f);
  G.assign((size_t)n * 2 * m, 0.f);
  for (int k = 0; k < m; ++k) {
    const double wgt = (k == 0 || 2 * k == n) ? 1.0 / n : 2.0 / n;
    for (int l = 0; l < n; ++l) {
      const double a = 2.0 * PI * (double)k * l / n;
      F[(size_t)k * n + l] = (float)std::cos(a);
      F[(size_t)(m + k) * n + l] = (float)(-std::sin(a));
      G[(size_t)l * 2 * m + k] = (float)(wgt * std::cos(a));
      G[(size_t)l * 2 * m + m + k] = (float)(-wgt * std::sin(a));
    }
  }
}

// splitmix64-driven normal deviates for the initial weights
struct Rng {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() { return std::sqrt(-2.0 * std::log(uniform())) * std::cos(2.0 * PI * uniform()); }
};

sft_status forward(sfs_handle h, const float* x, const float* p, int nb) {
  const int C = h->C, M = h->M;
  const long long ntok = (long long)nb * NTOK;
  // rotation layer r = phase(x F^T) G^T, by FFT per map row (FP32)
  rot_angle_kernel<<<grid_for((long long)nb * H), 256, 0, h->stream>>>(p, nb * H, h->alpha);
  rot_fft_kernel<<<(nb * H + 3) / 4, 256, 0, h->stream>>>(x, h->alpha, h->tw, nb * H, h->R);
  embed_kernel<<<grid_for(ntok), 256, 0, h->stream>>>(x, h->R, p, nb, h->E);
  h->kernels += 3;
  sft_status st = gemm(h, (int)ntok, C, KE, opnd(h->E, KE, 0, KMAJ), opnd(h->P + h->oWe, C, 0, MNMAJ), h->Hs[0], C, 0,
                       1.f, 0.f, h->P + h->obe, 1);
  if (st != SFT_OK) return st;
  for (int l = 0; l < h->L; ++l) {
    float* hcur = h->Hs[l];
    // Hh_bi = Fm h_bi (batched over b*HT + i)
    st = gemm(h, 2 * M, C, WT, opnd(h->Fm, WT, 0, KMAJ), opnd(hcur, C, (long long)WT * C, MNMAJ), h->Hh[l], C,
              (long long)2 * M * C, 1.f, 0.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    spectral_fwd_kernel<<<grid_for((long long)nb * HT * M * C), 256, 0, h->stream>>>(h->Hh[l], h->P + h->ow[l], nb,
                                                                                      M, C, h->Yh);
    h->kernels += 1;
    SFS_CUDA(cudaMemcpyAsync(h->U[l], hcur, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, WT, C, 2 * M, opnd(h->Gm, 2 * M, 0, KMAJ), opnd(h->Yh, C, (long long)2 * M * C, MNMAJ), h->U[l], C,
              (long long)WT * C, 1.f, 1.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, 2 * C, C, opnd(h->U[l], C, 0, KMAJ), opnd(h->P + h->oW1[l], 2 * C, 0, MNMAJ), h->Z[l],
              2 * C, 0, 1.f, 0.f, h->P + h->ob1[l], 1);
    if (st != SFT_OK) return st;
    gelu_fwd_kernel<<<grid_for(ntok * 2 * C), 256, 0, h->stream>>>(h->Z[l], ntok * 2 * C, h->A[l]);
    h->kernels += 1;
    SFS_CUDA(cudaMemcpyAsync(h->Hs[l + 1], h->U[l], ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, (int)ntok, C, 2 * C, opnd(h->A[l], 2 * C, 0, KMAJ), opnd(h->P + h->oW2[l], C, 0, MNMAJ),
              h->Hs[l + 1], C, 0, 1.f, 1.f, h->P + h->ob2[l], 1);
    if (st != SFT_OK) return st;
  }
  st = gemm(h, (int)ntok, 16, C, opnd(h->Hs[h->L], C, 0, KMAJ), opnd(h->P + h->oWd, 16, 0, MNMAJ), h->D, 16, 0, 1.f,
            0.f, h->P + h->obd, 1);
  if (st != SFT_OK) return st;
  // x_next = r + s (delta - <delta>_A): the correction carries no net flux
  unpatch_kernel<<<grid_for((long long)nb * H * W), 256, 0, h->stream>>>(h->D, nb, h->XN);
  flux_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->area, h->mpart);
  fold_map_sums<<<nb, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->msum);
  center_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->R, h->msum, h->area_total, nb);
  h->kernels += 4;
  SFS_CUDA(cudaGetLastError());
  return SFT_OK;
}

// Inference forward of the fused kernel (sfs_fused.cu): rotation by FFT,
// then one persistent kernel for embedding, blocks and decoder, then the
// flux-free centring.
sft_status forward_fused(sfs_handle h, const float* x, const float* p, int nb) {
  rot_angle_kernel<<<grid_for((long long)nb * H), 256, 0, h->stream>>>(p, nb * H, h->alpha);
  rot_fft_kernel<<<(nb * H + 3) / 4, 256, 0, h->stream>>>(x, h->alpha, h->tw, nb * H, h->R);
  h->kernels += 2;
  if (h->img_pver != h->pver) {
    SFS_CUDA(sfs_fused::build_image(h->P, h->po, h->L, h->Fm, h->Gm, h->img, h->stream));
    h->img_pver = h->pver;
    h->kernels += 1;
  }
  const int sms = (h->sm_budget > 0 && h->sm_budget < h->n_sm) ? h->sm_budget : h->n_sm;
  SFS_CUDA(sfs_fused::forward(h->img, h->L, h->P, h->po, x, h->R, p, nb, h->XN, sms, h->stream));
  h->kernels += 1;
  h->flops += 2.0 * nb * NTOK *
              ((double)KE * h->C + h->L * (2.0 * 2 * h->M * h->C + 2.0 * 2 * h->C * h->C) + 16.0 * h->C);
  flux_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->area, h->mpart);
  fold_map_sums<<<nb, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->msum);
  center_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->R, h->msum, h->area_total, nb);
  h->kernels += 3;
  SFS_CUDA(cudaGetLastError());
  return SFT_OK;
}

// Loss sums (into h->sums) and all parameter gradients (into h->G).
sft_status backward(sfs_handle h, const float* y, int nb) {
  const int C = h->C, M = h->M;
  const long long ntok = (long long)nb * NTOK;
  loss_sums_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, y, h->mpart);
  fold_map_sums<<<nb, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 3, h->lsum);
  loss_grad_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, y, h->lsum, h->area,
                                                                          h->area_total, nb, h->dD);
  h->kernels += 3;
  SFS_CUDA(cudaGetLastError());
  // decoder
  sft_status st = gemm_wgrad(h, C, 16, (int)ntok, opnd(h->Hs[h->L], C, 0, MNMAJ), opnd(h->dD, 16, 0, MNMAJ),
                             h->G + h->oWd);
  if (st != SFT_OK) return st;
  st = bias_grad(h, h->dD, ntok, 16, h->G + h->obd);
  if (st != SFT_OK) return st;
  st = gemm(h, (int)ntok, C, 16, opnd(h->dD, 16, 0, KMAJ), opnd(h->P + h->oWd, 16, 0, KMAJ), h->dH, C, 0, 1.f, 0.f,
            nullptr, 1);
  if (st != SFT_OK) return st;
  for (int l = h->L - 1; l >= 0; --l) {
    // h_{l+1} = u + a W2 + b2
    SFS_CUDA(cudaMemcpyAsync(h->dU, h->dH, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm_wgrad(h, 2 * C, C, (int)ntok, opnd(h->A[l], 2 * C, 0, MNMAJ), opnd(h->dH, C, 0, MNMAJ), h->G + h->oW2[l]);
    if (st != SFT_OK) return st;
    st = bias_grad(h, h->dH, ntok, C, h->G + h->ob2[l]);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, 2 * C, C, opnd(h->dH, C, 0, KMAJ), opnd(h->P + h->oW2[l], C, 0, KMAJ), h->dA, 2 * C, 0,
              1.f, 0.f, nullptr, 1);
    if (st != SFT_OK) return st;
    gelu_bwd_kernel<<<grid_for(ntok * 2 * C), 256, 0, h->stream>>>(h->dA, h->Z[l], ntok * 2 * C, h->dZ);
    h->kernels += 1;
    st = gemm_wgrad(h, C, 2 * C, (int)ntok, opnd(h->U[l], C, 0, MNMAJ), opnd(h->dZ, 2 * C, 0, MNMAJ),
                    h->G + h->oW1[l]);
    if (st != SFT_OK) return st;
    st = bias_grad(h, h->dZ, ntok, 2 * C, h->G + h->ob1[l]);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, C, 2 * C, opnd(h->dZ, 2 * C, 0, KMAJ), opnd(h->P + h->oW1[l], 2 * C, 0, KMAJ), h->dU, C,
              0, 1.f, 1.f, nullptr, 1);
    if (st != SFT_OK) return st;
    // u = h + Gm (w (.) Fm h)
    st = gemm(h, 2 * M, C, WT, opnd(h->Gm, 2 * M, 0, MNMAJ), opnd(h->dU, C, (long long)WT * C, MNMAJ), h->dYh, C,
              (long long)2 * M * C, 1.f, 0.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    spectral_bwd_w_kernel<<<grid_for((long long)HT * M * C), 256, 0, h->stream>>>(h->dYh, h->Hh[l], nb, M, C,
                                                                                  h->G + h->ow[l]);
    spectral_bwd_x_kernel<<<grid_for((long long)nb * HT * M * C), 256, 0, h->stream>>>(h->dYh, h->P + h->ow[l], nb,
                                                                                        M, C, h->dHh);
    h->kernels += 2;
    SFS_CUDA(cudaMemcpyAsync(h->dH, h->dU, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, WT, C, 2 * M, opnd(h->Fm, WT, 0, MNMAJ), opnd(h->dHh, C, (long long)2 * M * C, MNMAJ), h->dH, C,
              (long long)WT * C, 1.f, 1.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
  }
  st = gemm_wgrad(h, KE, C, (int)ntok, opnd(h->E, KE, 0, MNMAJ), opnd(h->dH, C, 0, MNMAJ), h->G + h->oWe);
  if (st != SFT_OK) return st;
  st = bias_grad(h, h->dH, ntok, C, h->G + h->obe);
  if (st != SFT_OK) return st;
  SFS_CUDA(cudaGetLastError());
  return SFT_OK;
}

sft_status check_batch(sfs_handle h, const void* a, const void* b, int n) {
  if (!h) return fail("NULL handle", SFT_ERR_ARG);
  if (!a || !b) return fail("NULL argument", SFT_ERR_ARG);
  if ((reinterpret_cast<uintptr_t>(a) & 15) != 0) return fail("maps must be 16-byte aligned", SFT_ERR_ARG);
  if (n <= 0 || n > h->maxb) return fail("batch size out of range", SFT_ERR_ARG);
  return SFT_OK;
}

// maps of the reductions: any count, in chunks of max_batch
sft_status check_maps(sfs_handle h, const void* a, const void* b, int n) {
  if (!h) return fail("NULL handle", SFT_ERR_ARG);
  if (!a || !b) return fail("NULL argument", SFT_ERR_ARG);
  if ((reinterpret_cast<uintptr_t>(a) & 15) != 0 || (reinterpret_cast<uintptr_t>(b) & 15) != 0)
    return fail("maps must be 16-byte aligned", SFT_ERR_ARG);
  if (n <= 0) return fail("map count out of range", SFT_ERR_ARG);
  return SFT_OK;
}

// pinned host staging of at least n doubles (grown between calls: every call
// that uses it ends with a stream synchronisation)
sft_status stage_host(sfs_handle h, long long n) {
  if (n <= h->hbig_n) return SFT_OK;
  if (h->hbig) cudaFreeHost(h->hbig);
  h->hbig = nullptr;
  h->hbig_n = 0;
  if (cudaMallocHost(&h->hbig, n * sizeof(double)) != cudaSuccess) return fail("pinned alloc failed", SFT_ERR_OOM);
  h->hbig_n = n;
  return SFT_OK;
}

float host_loss(sfs_handle h, int nb) {
  double l = 0.0;
  for (int b = 0; b < nb; ++b) l += h->hlsum[3 * b] / h->hlsum[3 * b + 1];
  return (float)(l / nb);
}

}  // namespace

extern "C" {

sft_status sfs_create(const sfs_config* cfg, void* cuda_stream, sfs_handle* out) {
  if (!cfg || !out) return fail("NULL argument", SFT_ERR_ARG);
  *out = nullptr;
  if (cfg->channels < 16 || cfg->channels % 16 || cfg->modes < 1 || cfg->modes > 64 || cfg->blocks < 1 ||
      cfg->blocks > 16 || cfg->max_batch < 1 || cfg->max_batch > 512)
    return fail("bad surrogate configuration", SFT_ERR_ARG);
  sfs_handle h = new sfs_net();
  h->C = cfg->channels;
  h->M = cfg->modes;
  h->L = cfg->blocks;
  h->maxb = cfg->max_batch;
  auto bail = [&](sft_status st) {
    sfs_destroy(h);
    return st;
  };
#define CR(x)                        \
  do {                               \
    sft_status s_ = (x);             \
    if (s_ != SFT_OK) return bail(s_); \
  } while (0)
  if (cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreate(&h->stream) != cudaSuccess) return bail(fail("cudaStreamCreate failed"));
    h->own_stream = true;
  }
  const int C = h->C, M = h->M, L = h->L;
  long long o = 0;
  auto take = [&](long long n) {
    const long long r = o;
    o += n;
    return r;
  };
  h->oWe = take((long long)KE * C);
  h->obe = take(C);
  h->oWd = take((long long)C * 16);
  h->obd = take(16);
  for (int l = 0; l < L; ++l) {
    h->ow.push_back(take((long long)HT * M * C * 2));
    h->oW1.push_back(take((long long)C * 2 * C));
    h->ob1.push_back(take(2 * C));
    h->oW2.push_back(take((long long)2 * C * C));
    h->ob2.push_back(take(C));
  }
  h->np = o;
  CR(dalloc(h, &h->P, h->np));
  CR(dalloc(h, &h->G, h->np));
  CR(dalloc(h, &h->Mo, h->np));
  CR(dalloc(h, &h->Vo, h->np));
  // initial weights (same scheme as the reference's init_params, own RNG)
  {
    std::vector<float> w(h->np, 0.f);
    Rng rng{cfg->seed};
    for (long long i = 0; i < (long long)39 * C; ++i) w[h->oWe + i] = (float)(rng.normal() / std::sqrt(39.0));
    for (long long i = 0; i < (long long)C * 16; ++i) w[h->oWd + i] = (float)(rng.normal() * 0.02 / std::sqrt((double)C));
    for (int l = 0; l < L; ++l) {
      for (long long i = 0; i < (long long)HT * M * C; ++i) {
        w[h->ow[l] + 2 * i] = (float)(0.5 + 0.02 * rng.normal());
        w[h->ow[l] + 2 * i + 1] = (float)(0.02 * rng.normal());
      }
      for (long long i = 0; i < (long long)C * 2 * C; ++i) w[h->oW1[l] + i] = (float)(rng.normal() / std::sqrt((double)C));
      for (long long i = 0; i < (long long)2 * C * C; ++i)
        w[h->oW2[l] + i] = (float)(rng.normal() * 0.5 / std::sqrt(2.0 * C));
    }
    if (cudaMemcpy(h->P, w.data(), h->np * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail("weight upload failed"));
    if (cudaMemset(h->Mo, 0, h->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(h->Vo, 0, h->np * sizeof(float)) != cudaSuccess)
      return bail(fail("moment init failed"));
  }
  // fixed matrices
  {
    std::vector<float> F, G;
    std::vector<float2> tw(W / 2);
    for (int j = 0; j < W / 2; ++j) {
      const double a = -2.0 * PI * j / W;
      tw[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    CR(dalloc(h, &h->tw, (long long)tw.size()));
    if (cudaMemcpy(h->tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail("twiddle upload failed"));
    dft_host(WT, M, F, G);
    CR(dalloc(h, &h->Fm, (long long)F.size()));
    CR(dalloc(h, &h->Gm, (long long)G.size()));
    if (cudaMemcpy(h->Fm, F.data(), F.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(h->Gm, G.data(), G.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail("dft upload failed"));
  }
  const long long nb = h->maxb, ntok = nb * NTOK;
  CR(dalloc(h, &h->R, nb * H * W));
  CR(dalloc(h, &h->XN, nb * H * W));
  CR(dalloc(h, &h->E, ntok * KE));
  CR(dalloc(h, &h->D, ntok * 16));
  h->Hs.assign(L + 1, nullptr);
  h->Hh.assign(L, nullptr);
  h->U.assign(L, nullptr);
  h->Z.assign(L, nullptr);
  h->A.assign(L, nullptr);
  for (int l = 0; l <= L; ++l) CR(dalloc(h, &h->Hs[l], ntok * C));
  for (int l = 0; l < L; ++l) {
    CR(dalloc(h, &h->Hh[l], nb * HT * 2 * M * C));
    CR(dalloc(h, &h->U[l], ntok * C));
    CR(dalloc(h, &h->Z[l], ntok * 2 * C));
    CR(dalloc(h, &h->A[l], ntok * 2 * C));
  }
  CR(dalloc(h, &h->Yh, nb * HT * 2 * M * C));
  CR(dalloc(h, &h->dD, ntok * 16));
  CR(dalloc(h, &h->dH, ntok * C));
  CR(dalloc(h, &h->dU, ntok * C));
  CR(dalloc(h, &h->dA, ntok * 2 * C));
  CR(dalloc(h, &h->dZ, ntok * 2 * C));
  CR(dalloc(h, &h->dYh, nb * HT * 2 * M * C));
  CR(dalloc(h, &h->dHh, nb * HT * 2 * M * C));
  h->part_elems = ((ntok + 1023) / 1024) * (long long)std::max(2 * C * C, KE * C);
  CR(dalloc(h, &h->part, h->part_elems));
  CR(dalloc(h, &h->gerr, 1));
  if (cudaMemsetAsync(h->gerr, 0, sizeof(int), h->stream) != cudaSuccess) return bail(fail("memset failed"));
  if (sfs_gemm::prepare() != cudaSuccess) return bail(fail("tensor-core GEMM: shared-memory limit not granted"));
  CR(dalloc(h, &h->sums, 2 * nb));
  CR(dalloc(h, &h->alpha, nb * H));
  CR(dalloc(h, &h->msum, 2 * nb));
  CR(dalloc(h, &h->mpart, nb * kRedBlocks * 3));
  CR(dalloc(h, &h->lsum, 3 * nb));
  {
    std::vector<double> ar(H);
    const double dth = PI / (H - 1), dph = 2.0 * PI / W;
    for (int j = 0; j < H; ++j)
      ar[j] = (j == 0 || j == H - 1) ? 2.0 * PI * (1.0 - std::cos(0.5 * dth)) / W : std::sin(j * dth) * dth * dph;
    CR(dalloc(h, &h->area, H));
    for (int j = 0; j < H; ++j) h->area_total += ar[j] * W;
    if (cudaMemcpy(h->area, ar.data(), H * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail("area upload failed"));
  }
  if (cudaMallocHost(&h->hlsum, 3 * nb * sizeof(double)) != cudaSuccess) return bail(fail("pinned alloc failed"));
  if (cudaMallocHost(&h->hgerr, sizeof(int)) != cudaSuccess) return bail(fail("pinned alloc failed"));
  *h->hgerr = 0;
  h->fused = C == sfs_fused::kChannels && M == sfs_fused::kModes && L <= sfs_fused::kMaxBlocks;
  if (h->fused) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return bail(fail("device query failed"));
    if (sfs_fused::prepare(L) != cudaSuccess) return bail(fail("fused forward: shared-memory limit not granted"));
    CR(dalloc(h, &h->img, (long long)sfs_fused::image_bytes(L)));
    h->po.We = h->oWe;
    h->po.be = h->obe;
    h->po.Wd = h->oWd;
    h->po.bd = h->obd;
    for (int l = 0; l < L; ++l) {
      h->po.w[l] = h->ow[l];
      h->po.W1[l] = h->oW1[l];
      h->po.b1[l] = h->ob1[l];
      h->po.W2[l] = h->oW2[l];
      h->po.b2[l] = h->ob2[l];
    }
  }
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(fail("create sync failed"));
#undef CR
  *out = h;
  return SFT_OK;
}

sft_status sfs_destroy(sfs_handle h) {
  if (!h) return SFT_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->allocs) cudaFree(p);
  if (h->hlsum) cudaFreeHost(h->hlsum);
  if (h->hgerr) cudaFreeHost(h->hgerr);
  if (h->hbig) cudaFreeHost(h->hbig);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return SFT_OK;
}

int64_t sfs_num_params(sfs_handle h) { return h ? h->np : 0; }

sft_status sfs_set_sm_budget(sfs_handle h, int32_t n_sm) {
  if (!h) return fail("NULL handle", SFT_ERR_ARG);
  if (n_sm < 0) return fail("SM budget must be >= 0", SFT_ERR_ARG);
  h->sm_budget = n_sm;
  return SFT_OK;
}

sft_status sfs_debug_gemm(sfs_handle h, int32_t M, int32_t N, int32_t K, const void* A, int32_t a_bf16,
                          int32_t a_mn_major, int64_t lda, int64_t sA, const void* B, int32_t b_bf16,
                          int32_t b_mn_major, int64_t ldb, int64_t sB, float* C, int64_t ldc, int64_t sC,
                          float alpha, float beta, const float* bias, int32_t kchunk, int32_t batch) {
  if (!h) return fail("NULL handle", SFT_ERR_ARG);
  if (!A || !B || !C) return fail("NULL argument", SFT_ERR_ARG);
  if (M <= 0 || N <= 0 || K < 0 || batch <= 0 || kchunk < 0) return fail("GEMM shape out of range", SFT_ERR_ARG);
  const sfs_gemm::Operand a{A, a_bf16 ? sfs_gemm::BF16 : sfs_gemm::F32, a_mn_major ? 1 : 0, lda, sA};
  const sfs_gemm::Operand b{B, b_bf16 ? sfs_gemm::BF16 : sfs_gemm::F32, b_mn_major ? 1 : 0, ldb, sB};
  const sfs_gemm::Problem pr{M, N, K, a, b, C, ldc, sC, alpha, beta, bias, kchunk, batch};
  const cudaError_t e = sfs_gemm::launch(pr, h->gerr, h->stream);
  if (e == cudaErrorInvalidValue) return fail("GEMM operands the kernel cannot take", SFT_ERR_ARG);
  SFS_CUDA(e);
  SFS_CUDA(cudaMemcpyAsync(h->hgerr, h->gerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  return check_gemm_error(h);
}

sft_status sfs_set_params(sfs_handle h, const float* host_params) {
  if (!h || !host_params) return fail("NULL argument", SFT_ERR_ARG);
  SFS_CUDA(cudaMemcpyAsync(h->P, host_params, h->np * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  SFS_CUDA(cudaMemsetAsync(h->Mo, 0, h->np * sizeof(float), h->stream));
  SFS_CUDA(cudaMemsetAsync(h->Vo, 0, h->np * sizeof(float), h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  h->t = 0;
  h->pver += 1;
  return SFT_OK;
}

sft_status sfs_get_params(sfs_handle h, float* host_params) {
  if (!h || !host_params) return fail("NULL argument", SFT_ERR_ARG);
  SFS_CUDA(cudaMemcpyAsync(host_params, h->P, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  return SFT_OK;
}

sft_status sfs_forward(sfs_handle h, const float* x, const float* p, int32_t n, float* y) {
  nvtxRangePushA("sfs_forward");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  sft_status st = check_batch(h, x, p, n);
  if (st != SFT_OK) return st;
  if (!y) return fail("NULL output", SFT_ERR_ARG);
  st = h->fused ? forward_fused(h, x, p, n) : forward(h, x, p, n);
  if (st != SFT_OK) return st;
  SFS_CUDA(cudaMemcpyAsync(y, h->XN, (size_t)n * H * W * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
  return SFT_OK;
}

sft_status sfs_loss_grad(sfs_handle h, const float* x, const float* p, const float* y, int32_t n, float* loss,
                         float* host_grad) {
  sft_status st = check_batch(h, x, p, n);
  if (st != SFT_OK) return st;
  if (!y || !loss || !host_grad) return fail("NULL argument", SFT_ERR_ARG);
  st = forward(h, x, p, n);
  if (st != SFT_OK) return st;
  st = backward(h, y, n);
  if (st != SFT_OK) return st;
  SFS_CUDA(cudaMemcpyAsync(h->hlsum, h->lsum, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaMemcpyAsync(host_grad, h->G, h->np * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaMemcpyAsync(h->hgerr, h->gerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  st = check_gemm_error(h);
  if (st != SFT_OK) return st;
  *loss = host_loss(h, n);
  return SFT_OK;
}

sft_status sfs_train_step(sfs_handle h, const float* x, const float* p, const float* y, int32_t n, double lr,
                          double wd, float* loss) {
  nvtxRangePushA("sfs_train_step");
  struct Pop {
    ~Pop() { nvtxRangePop(); }
  } pop;
  sft_status st = check_batch(h, x, p, n);
  if (st != SFT_OK) return st;
  if (!y) return fail("NULL argument", SFT_ERR_ARG);
  st = forward(h, x, p, n);
  if (st != SFT_OK) return st;
  st = backward(h, y, n);
  if (st != SFT_OK) return st;
  h->t += 1;
  const float bc1 = (float)(1.0 - std::pow(0.9, h->t)), bc2 = (float)(1.0 - std::pow(0.999, h->t));
  adamw_kernel<<<grid_for(h->np), 256, 0, h->stream>>>(h->P, h->G, h->Mo, h->Vo, h->np, (float)lr, (float)wd, bc1,
                                                       bc2);
  h->kernels += 1;
  h->pver += 1;
  SFS_CUDA(cudaGetLastError());
  if (loss) {
    SFS_CUDA(cudaMemcpyAsync(h->hlsum, h->lsum, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    SFS_CUDA(cudaMemcpyAsync(h->hgerr, h->gerr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    SFS_CUDA(cudaStreamSynchronize(h->stream));
    st = check_gemm_error(h);
    if (st != SFT_OK) return st;
    *loss = host_loss(h, n);
  }
  return SFT_OK;
}

sft_status sfs_rel_l2(sfs_handle h, const float* a, const float* b, int32_t n, double* out) {
  sft_status st = check_maps(h, a, b, n);
  if (st != SFT_OK) return st;
  if (!out) return fail("NULL output", SFT_ERR_ARG);
  st = stage_host(h, 2 * (long long)n);
  if (st != SFT_OK) return st;
  for (int c0 = 0; c0 < n; c0 += h->maxb) {  // chunks of max_batch maps, one synchronisation
    const int m = std::min(h->maxb, n - c0);
    const long long off = (long long)c0 * H * W;
    sumsq_kernel<<<dim3(kRedBlocks, m), 256, 0, h->stream>>>(a + off, b + off, m, h->mpart);
    fold_map_sums<<<m, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->sums);
    h->kernels += 2;
    SFS_CUDA(cudaGetLastError());
    SFS_CUDA(cudaMemcpyAsync(h->hbig + 2 * c0, h->sums, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < n; ++i) out[i] = std::sqrt(h->hbig[2 * i] / h->hbig[2 * i + 1]);
  return SFT_OK;
}

sft_status sfs_flux(sfs_handle h, const float* maps, int32_t n, double* out) {
  sft_status st = check_maps(h, maps, maps, n);
  if (st != SFT_OK) return st;
  if (!out) return fail("NULL output", SFT_ERR_ARG);
  st = stage_host(h, 2 * (long long)n);
  if (st != SFT_OK) return st;
  for (int c0 = 0; c0 < n; c0 += h->maxb) {
    const int m = std::min(h->maxb, n - c0);
    flux_kernel<<<dim3(kRedBlocks, m), 256, 0, h->stream>>>(maps + (long long)c0 * H * W, h->area, h->mpart);
    fold_map_sums<<<m, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->sums);
    h->kernels += 2;
    SFS_CUDA(cudaGetLastError());
    SFS_CUDA(cudaMemcpyAsync(h->hbig + 2 * c0, h->sums, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  }
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->hbig, 2 * (size_t)n * sizeof(double));
  return SFT_OK;
}

sft_status sfs_counters(sfs_handle h, int64_t* gemm_launches, double* gemm_flops, int64_t* kernel_launches) {
  if (!h) return fail("NULL handle", SFT_ERR_ARG);
  if (gemm_launches) *gemm_launches = h->gemms;
  if (gemm_flops) *gemm_flops = h->flops;
  if (kernel_launches) *kernel_launches = h->kernels;
  return SFT_OK;
}

}  // extern "C"
