// sfs.cu -- the learned one-day surrogate (include/sfs.h): BF16 tensor-core
// GEMMs with FP32 accumulation, the network's forward and backward passes,
// AdamW, and the C-ABI.
//
// GEMM: mma.sync m16n8k16 (BF16 x BF16 -> FP32) on 128 x 64 x 32 block
// tiles, operands converted from FP32 to BF16 as they are staged in shared
// memory and fed to the tensor cores with ldmatrix; batched (strides, a
// zero stride shares an operand), transposes by layout flags, split-K for
// the weight gradients (K = batch x tokens), and a split-BF16 mode (hi*hi +
// hi*lo + lo*hi) for products that must stay ~FP32-accurate.  The fixed
// rotation layer is an FFT per map row (rot_fft_kernel), not a GEMM.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "sfs.h"
#include "sfs_fused.cuh"
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

// ---------------------------------------------------------------------------
// GEMM
// ---------------------------------------------------------------------------
struct GemmArgs {
  int M, N, K;
  const float* A;
  long long lda, sA;
  int tA;  // 0: A[m*lda + k]; 1: A[k*lda + m]
  const float* B;
  long long ldb, sB;
  int tB;  // 0: B[k*ldb + n]; 1: B[n*ldb + k]
  float* C;
  long long ldc, sC;
  float alpha, beta;
  const float* bias;  // per column, may be null
  int kchunk;         // > 0: batch b covers k in [b*kchunk, (b+1)*kchunk) (split-K)
  int vecA, vecB;     // float4 loads allowed along the contiguous dimension
};

constexpr int BM = 128, BN = 64, BK = 32, PADK = 8;

__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  const uint32_t a = static_cast<uint32_t>(__cvta_generic_to_shared(p));
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Global -> register staging of one k-tile: A is BM x BK, B is BK x BN, 16
// and 8 values per thread, as float4 along the contiguous dimension when the
// layout and alignment allow it (vecA / vecB), else element by element.
struct Stage {
  float a[16], b[8];
};

__device__ __forceinline__ void load_tile(const GemmArgs& g, const float* A, const float* Bm, int m0, int n0, int k0,
                                          int kb1, Stage& st) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int v = tid + q * 256;  // float4 index within the tile
    int m, k;
    if (!g.tA) { m = v >> 3; k = (v & 7) * 4; } else { k = v >> 5; m = (v & 31) * 4; }
    const int gm = m0 + m, gk = k0 + k;
    if (!g.tA) {
      if (g.vecA && gm < g.M && gk + 3 < kb1) {
        const float4 t = *reinterpret_cast<const float4*>(A + (long long)gm * g.lda + gk);
        st.a[4 * q] = t.x; st.a[4 * q + 1] = t.y; st.a[4 * q + 2] = t.z; st.a[4 * q + 3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          st.a[4 * q + e] = (gm < g.M && gk + e < kb1) ? A[(long long)gm * g.lda + gk + e] : 0.f;
      }
    } else {
      if (g.vecA && gm + 3 < g.M && gk < kb1) {
        const float4 t = *reinterpret_cast<const float4*>(A + (long long)gk * g.lda + gm);
        st.a[4 * q] = t.x; st.a[4 * q + 1] = t.y; st.a[4 * q + 2] = t.z; st.a[4 * q + 3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          st.a[4 * q + e] = (gm + e < g.M && gk < kb1) ? A[(long long)gk * g.lda + gm + e] : 0.f;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int v = tid + q * 256;
    int n, k;
    if (!g.tB) { k = v >> 4; n = (v & 15) * 4; } else { n = v >> 3; k = (v & 7) * 4; }
    const int gn = n0 + n, gk = k0 + k;
    if (!g.tB) {
      if (g.vecB && gn + 3 < g.N && gk < kb1) {
        const float4 t = *reinterpret_cast<const float4*>(Bm + (long long)gk * g.ldb + gn);
        st.b[4 * q] = t.x; st.b[4 * q + 1] = t.y; st.b[4 * q + 2] = t.z; st.b[4 * q + 3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          st.b[4 * q + e] = (gn + e < g.N && gk < kb1) ? Bm[(long long)gk * g.ldb + gn + e] : 0.f;
      }
    } else {
      if (g.vecB && gn < g.N && gk + 3 < kb1) {
        const float4 t = *reinterpret_cast<const float4*>(Bm + (long long)gn * g.ldb + gk);
        st.b[4 * q] = t.x; st.b[4 * q + 1] = t.y; st.b[4 * q + 2] = t.z; st.b[4 * q + 3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
          st.b[4 * q + e] = (gn < g.N && gk + e < kb1) ? Bm[(long long)gn * g.ldb + gk + e] : 0.f;
      }
    }
  }
}

template <bool SPLIT>
__device__ __forceinline__ void store_tile(const GemmArgs& g, const Stage& st,
                                           __nv_bfloat16 (*sA)[BM][BK + PADK], __nv_bfloat16 (*sB)[BN][BK + PADK]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int v = tid + q * 256;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int m, k;
      if (!g.tA) { m = v >> 3; k = (v & 7) * 4 + e; } else { k = v >> 5; m = (v & 31) * 4 + e; }
      const float x = st.a[4 * q + e];
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      sA[0][m][k] = hi;
      if (SPLIT) sA[1][m][k] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int v = tid + q * 256;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int n, k;
      if (!g.tB) { k = v >> 4; n = (v & 15) * 4 + e; } else { n = v >> 3; k = (v & 7) * 4 + e; }
      const float x = st.b[4 * q + e];
      const __nv_bfloat16 hi = __float2bfloat16_rn(x);
      sB[0][n][k] = hi;
      if (SPLIT) sB[1][n][k] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
  }
}

template <bool SPLIT>
__global__ void __launch_bounds__(256) gemm_kernel(GemmArgs g) {
  constexpr int NS = SPLIT ? 2 : 1;
  __shared__ __align__(16) __nv_bfloat16 sA[NS][BM][BK + PADK];
  __shared__ __align__(16) __nv_bfloat16 sB[NS][BN][BK + PADK];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;  // 4 x 2 warps, 32 x 32 each
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN, b = blockIdx.z;
  const float* A = g.A + (g.kchunk ? 0 : b * g.sA);
  const float* Bm = g.B + (g.kchunk ? 0 : b * g.sB);
  float* C = g.C + b * g.sC;
  const int kb0 = g.kchunk ? b * g.kchunk : 0;
  const int kb1 = g.kchunk ? min(g.K, kb0 + g.kchunk) : g.K;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  (void)tid;
  Stage st;
  if (kb0 < kb1) load_tile(g, A, Bm, m0, n0, kb0, kb1, st);
  for (int k0 = kb0; k0 < kb1; k0 += BK) {
    store_tile<SPLIT>(g, st, sA, sB);
    __syncthreads();
    // the next tile's global loads are in flight while the tensor cores work
    if (k0 + BK < kb1) load_tile(g, A, Bm, m0, n0, k0 + BK, kb1, st);
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t af[NS][2][4], bf[NS][4][2];
#pragma unroll
      for (int s = 0; s < NS; ++s) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
          ldsm_x4(af[s][mt], &sA[s][wm * 32 + mt * 16 + (lane & 15)][kk + (lane >> 4) * 8]);
#pragma unroll
        for (int np2 = 0; np2 < 2; ++np2) {
          uint32_t r[4];
          ldsm_x4(r, &sB[s][wn * 32 + np2 * 16 + (lane & 7) + ((lane >> 4) << 3)][kk + ((lane >> 3) & 1) * 8]);
          bf[s][np2 * 2][0] = r[0];
          bf[s][np2 * 2][1] = r[1];
          bf[s][np2 * 2 + 1][0] = r[2];
          bf[s][np2 * 2 + 1][1] = r[3];
        }
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          mma16816(acc[mt][nt], af[0][mt], bf[0][nt][0], bf[0][nt][1]);
          if (SPLIT) {
            mma16816(acc[mt][nt], af[0][mt], bf[NS - 1][nt][0], bf[NS - 1][nt][1]);
            mma16816(acc[mt][nt], af[NS - 1][mt], bf[0][nt][0], bf[0][nt][1]);
          }
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + wm * 32 + mt * 16 + (lane >> 2) + (q >= 2 ? 8 : 0);
        const int col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2 + (q & 1);
        if (row < g.M && col < g.N) {
          float* cp = C + (long long)row * g.ldc + col;
          float v = g.alpha * acc[mt][nt][q];
          if (g.beta != 0.f) v += g.beta * *cp;
          if (g.bias) v += g.bias[col];
          *cp = v;
        }
      }
}

// out[i] = beta * out[i] + sum_s part[s * n + i]
__global__ void splitk_reduce(const float* __restrict__ part, int ns, long long n, float beta,
                              float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int q = 0; q < ns; ++q) s += part[q * n + i];
    out[i] = (beta != 0.f ? beta * out[i] : 0.f) + s;
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

// Layer R by FFT, one block of 256 threads per map row: the 512-point DFT of
// the real row (radix-2 in shared memory: decimation in time from a
// bit-reversed load), Y_k = X_k exp(-i k alpha_row) on modes 0..256, the
// Hermitian extension Z_{512-k} = conj(Y_k) (the Nyquist mode keeps its real
// part only, as the truncated synthesis G does), and the inverse transform
// (decimation in frequency, conjugate twiddles) scaled by 1/512.  The same map
// as r = phase(x F^T) G^T, in FP32 with O(log n) rounding.
// tw[j] = exp(-2 pi i j / 512), j < 256.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(256) rot_fft_kernel(const float* __restrict__ x, const double* __restrict__ alpha,
                                                      const float2* __restrict__ tw, float* __restrict__ r) {
  static_assert(W == 512, "rot_fft_kernel is written for 512-point rows");
  __shared__ float2 s[W];
  const int row = blockIdx.x, t = threadIdx.x;
  const float* xr = x + (long long)row * W;
  s[__brev(t) >> 23] = make_float2(xr[t], 0.f);
  s[__brev(t + 256) >> 23] = make_float2(xr[t + 256], 0.f);
  __syncthreads();
  for (int half = 1; half < W; half <<= 1) {  // DIT stages
    const int pos = t & (half - 1), i0 = ((t - pos) << 1) + pos, i1 = i0 + half;
    const float2 u = s[i0], v = cmul(s[i1], tw[pos * (256 / half)]);
    s[i0] = make_float2(u.x + v.x, u.y + v.y);
    s[i1] = make_float2(u.x - v.x, u.y - v.y);
    __syncthreads();
  }
  // phase on k = t (and k = 256 by thread 0); Z_{512-k} = conj(Y_k) lands in
  // slots 257..511, which no thread reads
  const double a = alpha[row];
  for (int k = t; k <= W / 2; k += 256) {
    const double ang = k * a;
    const double red = ang - (2.0 * PI) * rint(ang * (1.0 / (2.0 * PI)));  // in [-pi, pi]
    float sn, cs;
    sincosf((float)red, &sn, &cs);
    const float2 X = s[k];
    const float2 Y = make_float2(X.x * cs + X.y * sn, X.y * cs - X.x * sn);
    if (k == W / 2) {
      s[k] = make_float2(Y.x, 0.f);
    } else {
      s[k] = Y;
      if (k > 0) s[W - k] = make_float2(Y.x, -Y.y);
    }
  }
  __syncthreads();
  for (int half = W / 2; half >= 1; half >>= 1) {  // DIF stages, conjugate twiddles
    const int pos = t & (half - 1), i0 = ((t - pos) << 1) + pos, i1 = i0 + half;
    const float2 u = s[i0], v = s[i1];
    const float2 w = tw[pos * (256 / half)];
    s[i0] = make_float2(u.x + v.x, u.y + v.y);
    s[i1] = cmul(make_float2(u.x - v.x, u.y - v.y), make_float2(w.x, -w.y));
    __syncthreads();
  }
  float* rr = r + (long long)row * W;
  constexpr float inv = 1.0f / W;
  rr[t] = s[__brev(t) >> 23].x * inv;
  rr[t + 256] = s[__brev(t + 256) >> 23].x * inv;
}

// E[token][48]: 4x4 patches of x/s and r/s, normalised parameters, cos/sin of
// the patch-row colatitude, zeros.  One thread per token.
__global__ void embed_kernel(const float* __restrict__ x, const float* __restrict__ r,
                             const float* __restrict__ p, int nb, float* __restrict__ E) {
  const long long n = (long long)nb * NTOK;
  const float ref[5] = {13.38f, -2.30f, -1.62f, 15.0f, 500.0f};
  const float spr[5] = {1.338f, 0.230f, 0.162f, 5.0f, 250.0f};
  for (long long tok = blockIdx.x * (long long)blockDim.x + threadIdx.x; tok < n;
       tok += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(tok / NTOK), t = (int)(tok % NTOK);
    const int i = t / WT, l = t % WT;
    float4* out = reinterpret_cast<float4*>(E + tok * KE);
    const float inv = 1.0f / SCALE;
#pragma unroll
    for (int pr = 0; pr < PATCH; ++pr) {
      const long long off = ((long long)b * H + i * PATCH + pr) * W + l * PATCH;
      float4 vx = *reinterpret_cast<const float4*>(x + off);
      float4 vr = *reinterpret_cast<const float4*>(r + off);
      vx.x *= inv; vx.y *= inv; vx.z *= inv; vx.w *= inv;
      vr.x *= inv; vr.y *= inv; vr.z *= inv; vr.w *= inv;
      out[pr] = vx;
      out[4 + pr] = vr;
    }
    const float q0 = (p[5 * b + 0] - ref[0]) / spr[0], q1 = (p[5 * b + 1] - ref[1]) / spr[1];
    const float q2 = (p[5 * b + 2] - ref[2]) / spr[2], q3 = (p[5 * b + 3] - ref[3]) / spr[3];
    const float q4 = (p[5 * b + 4] - ref[4]) / spr[4];
    const double th = (i + 0.5) * PATCH * (PI / (H - 1));
    out[8] = make_float4(q0, q1, q2, q3);
    out[9] = make_float4(q4, (float)cos(th), (float)sin(th), 0.f);
    out[10] = make_float4(0.f, 0.f, 0.f, 0.f);
    out[11] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Yh = w (.) Hh per (latent row i, mode k, channel c); layout [(b*HT+i)][2M][C].
__global__ void spectral_fwd_kernel(const float* __restrict__ Hh, const float* __restrict__ w, int nb, int M,
                                    int C, float* __restrict__ Yh) {
  const long long n = (long long)nb * HT * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int k = (int)((e / C) % M);
    const long long bi = e / ((long long)C * M);
    const int i = (int)(bi % HT);
    const float* hp = Hh + bi * 2 * M * C;
    float* yp = Yh + bi * 2 * M * C;
    const float hr = hp[(long long)k * C + c], hi = hp[(long long)(M + k) * C + c];
    const float wr = w[(((long long)i * M + k) * C + c) * 2], wi = w[(((long long)i * M + k) * C + c) * 2 + 1];
    yp[(long long)k * C + c] = wr * hr - wi * hi;
    yp[(long long)(M + k) * C + c] = wr * hi + wi * hr;
  }
}

// dHh = conj-transpose action of w on dYh.
__global__ void spectral_bwd_x_kernel(const float* __restrict__ dYh, const float* __restrict__ w, int nb, int M,
                                      int C, float* __restrict__ dHh) {
  const long long n = (long long)nb * HT * M * C;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(e % C);
    const int k = (int)((e / C) % M);
    const long long bi = e / ((long long)C * M);
    const int i = (int)(bi % HT);
    const float* dp = dYh + bi * 2 * M * C;
    float* op = dHh + bi * 2 * M * C;
    const float dr = dp[(long long)k * C + c], di = dp[(long long)(M + k) * C + c];
    const float wr = w[(((long long)i * M + k) * C + c) * 2], wi = w[(((long long)i * M + k) * C + c) * 2 + 1];
    op[(long long)k * C + c] = wr * dr + wi * di;
    op[(long long)(M + k) * C + c] = -wi * dr + wr * di;
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

__global__ void gelu_fwd_kernel(const float* __restrict__ z, long long n, float* __restrict__ a) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    a[e] = gelu_f(z[e]);
}

__global__ void gelu_bwd_kernel(const float* __restrict__ da, const float* __restrict__ z, long long n,
                                float* __restrict__ dz) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    dz[e] = da[e] * gelu_g(z[e]);
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
  const long long n = (long long)nb * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / (H * W));
    const float mean = (float)(msum[2 * b] / area_total);
    xn[e] = r[e] + SCALE * (xn[e] - mean);
  }
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
// the centring: s (g - A_row sum(g) / sum(A)).
__global__ void loss_grad_kernel(const float* __restrict__ xn, const float* __restrict__ y,
                                 const double* __restrict__ sums, const double* __restrict__ area,
                                 double area_total, int nb, float* __restrict__ dd) {
  const long long n = (long long)nb * H * W;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(e / (H * W)), rem = (int)(e % (H * W));
    const int row = rem / W, col = rem % W;
    const long long tok = (long long)b * NTOK + (row / PATCH) * WT + col / PATCH;
    const double k = 2.0 / (sums[3 * b + 1] * nb);
    const double g = k * (double(xn[e]) - double(y[e]));
    const double gsum = k * sums[3 * b + 2];
    dd[tok * 16 + (row % PATCH) * PATCH + col % PATCH] = (float)(SCALE * (g - area[row] * gsum / area_total));
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

__global__ void fill_kernel(float* __restrict__ a, long long n, float v) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
    a[e] = v;
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
  float *Fm = nullptr, *Gm = nullptr, *ones = nullptr;
  float2* tw = nullptr;  // FFT twiddles exp(-2 pi i j / W), j < W/2
  // activations
  float *R = nullptr, *E = nullptr, *D = nullptr, *XN = nullptr;
  std::vector<float*> Hs, Hh, U, Z, A;
  float *Yh = nullptr;
  // gradients of activations
  float *dD = nullptr, *dH = nullptr, *dU = nullptr, *dA = nullptr, *dZ = nullptr, *dYh = nullptr, *dHh = nullptr;
  float* part = nullptr;
  long long part_elems = 0;
  double *sums = nullptr, *hsums = nullptr;
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

// float4 loads need 16-byte aligned rows: base, leading dimension and batch
// stride all multiples of four floats.
int vec_ok(const float* p, long long ld, long long stride) {
  return ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && ld % 4 == 0 && stride % 4 == 0) ? 1 : 0;
}

// C = alpha op(A) op(B) + beta C + bias, batched (strides) or split-K.
sft_status gemm(sfs_handle h, int M, int N, int K, const float* A, long long lda, long long sA, int tA,
                const float* B, long long ldb, long long sB, int tB, float* C, long long ldc, long long sC,
                float alpha, float beta, const float* bias, int batch, bool split = false) {
  GemmArgs g{M, N, K, A, lda, sA, tA, B, ldb, sB, tB, C, ldc, sC, alpha, beta, bias, 0,
             vec_ok(A, lda, sA), vec_ok(B, ldb, sB)};
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  if (split) gemm_kernel<true><<<grid, 256, 0, h->stream>>>(g);
  else gemm_kernel<false><<<grid, 256, 0, h->stream>>>(g);
  SFS_CUDA(cudaGetLastError());
  h->gemms += 1;
  h->kernels += 1;
  h->flops += 2.0 * M * N * (double)K * batch * (split ? 3 : 1);
  return SFT_OK;
}

// Weight gradient C[M][N] (ldc = N) = op(A) op(B) with a long K: split-K into
// partial products, then a fixed-order reduction.
sft_status gemm_wgrad(sfs_handle h, int M, int N, int K, const float* A, long long lda, int tA, const float* B,
                      long long ldb, int tB, float* C) {
  const int kchunk = 1024;
  const int ns = (K + kchunk - 1) / kchunk;
  if ((long long)ns * M * N > h->part_elems) return fail("split-K scratch too small", SFT_ERR_ARG);
  GemmArgs g{M, N, K, A, lda, 0, tA, B, ldb, 0, tB, h->part, N, (long long)M * N, 1.f, 0.f, nullptr, kchunk,
             vec_ok(A, lda, 0), vec_ok(B, ldb, 0)};
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, ns);
  gemm_kernel<false><<<grid, 256, 0, h->stream>>>(g);
  SFS_CUDA(cudaGetLastError());
  splitk_reduce<<<grid_for((long long)M * N), 256, 0, h->stream>>>(h->part, ns, (long long)M * N, 0.f, C);
  SFS_CUDA(cudaGetLastError());
  h->gemms += 1;
  h->kernels += 2;
  h->flops += 2.0 * M * N * (double)K;
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
  rot_fft_kernel<<<nb * H, 256, 0, h->stream>>>(x, h->alpha, h->tw, h->R);
  embed_kernel<<<grid_for(ntok), 256, 0, h->stream>>>(x, h->R, p, nb, h->E);
  h->kernels += 3;
  sft_status st = gemm(h, (int)ntok, C, KE, h->E, KE, 0, 0, h->P + h->oWe, C, 0, 0, h->Hs[0], C, 0, 1.f, 0.f, h->P + h->obe, 1);
  if (st != SFT_OK) return st;
  for (int l = 0; l < h->L; ++l) {
    float* hcur = h->Hs[l];
    // Hh_bi = Fm h_bi (batched over b*HT + i)
    st = gemm(h, 2 * M, C, WT, h->Fm, WT, 0, 0, hcur, C, (long long)WT * C, 0, h->Hh[l], C,
              (long long)2 * M * C, 1.f, 0.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    spectral_fwd_kernel<<<grid_for((long long)nb * HT * M * C), 256, 0, h->stream>>>(h->Hh[l], h->P + h->ow[l], nb,
                                                                                      M, C, h->Yh);
    h->kernels += 1;
    SFS_CUDA(cudaMemcpyAsync(h->U[l], hcur, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, WT, C, 2 * M, h->Gm, 2 * M, 0, 0, h->Yh, C, (long long)2 * M * C, 0, h->U[l], C, (long long)WT * C,
              1.f, 1.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, 2 * C, C, h->U[l], C, 0, 0, h->P + h->oW1[l], 2 * C, 0, 0, h->Z[l], 2 * C, 0, 1.f, 0.f,
              h->P + h->ob1[l], 1);
    if (st != SFT_OK) return st;
    gelu_fwd_kernel<<<grid_for(ntok * 2 * C), 256, 0, h->stream>>>(h->Z[l], ntok * 2 * C, h->A[l]);
    h->kernels += 1;
    SFS_CUDA(cudaMemcpyAsync(h->Hs[l + 1], h->U[l], ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, (int)ntok, C, 2 * C, h->A[l], 2 * C, 0, 0, h->P + h->oW2[l], C, 0, 0, h->Hs[l + 1], C, 0, 1.f, 1.f,
              h->P + h->ob2[l], 1);
    if (st != SFT_OK) return st;
  }
  st = gemm(h, (int)ntok, 16, C, h->Hs[h->L], C, 0, 0, h->P + h->oWd, 16, 0, 0, h->D, 16, 0, 1.f, 0.f,
            h->P + h->obd, 1);
  if (st != SFT_OK) return st;
  // x_next = r + s (delta - <delta>_A): the correction carries no net flux
  unpatch_kernel<<<grid_for((long long)nb * H * W), 256, 0, h->stream>>>(h->D, nb, h->XN);
  flux_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->area, h->mpart);
  fold_map_sums<<<nb, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->msum);
  center_kernel<<<grid_for((long long)nb * H * W), 256, 0, h->stream>>>(h->XN, h->R, h->msum, h->area_total, nb);
  h->kernels += 4;
  SFS_CUDA(cudaGetLastError());
  return SFT_OK;
}

// Inference forward of the fused kernel (sfs_fused.cu): rotation by FFT,
// then one persistent kernel for embedding, blocks and decoder, then the
// flux-free centring.
sft_status forward_fused(sfs_handle h, const float* x, const float* p, int nb) {
  rot_angle_kernel<<<grid_for((long long)nb * H), 256, 0, h->stream>>>(p, nb * H, h->alpha);
  rot_fft_kernel<<<nb * H, 256, 0, h->stream>>>(x, h->alpha, h->tw, h->R);
  h->kernels += 2;
  if (h->img_pver != h->pver) {
    SFS_CUDA(sfs_fused::build_image(h->P, h->po, h->L, h->Fm, h->Gm, h->img, h->stream));
    h->img_pver = h->pver;
    h->kernels += 1;
  }
  SFS_CUDA(sfs_fused::forward(h->img, h->L, h->P, h->po, x, h->R, p, nb, h->XN, h->n_sm, h->stream));
  h->kernels += 1;
  h->flops += 2.0 * nb * NTOK *
              ((double)KE * h->C + h->L * (2.0 * 2 * h->M * h->C + 2.0 * 2 * h->C * h->C) + 16.0 * h->C);
  flux_kernel<<<dim3(kRedBlocks, nb), 256, 0, h->stream>>>(h->XN, h->area, h->mpart);
  fold_map_sums<<<nb, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->msum);
  center_kernel<<<grid_for((long long)nb * H * W), 256, 0, h->stream>>>(h->XN, h->R, h->msum, h->area_total, nb);
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
  loss_grad_kernel<<<grid_for((long long)nb * H * W), 256, 0, h->stream>>>(h->XN, y, h->lsum, h->area,
                                                                          h->area_total, nb, h->dD);
  h->kernels += 3;
  SFS_CUDA(cudaGetLastError());
  // decoder
  sft_status st = gemm_wgrad(h, C, 16, (int)ntok, h->Hs[h->L], C, 1, h->dD, 16, 0, h->G + h->oWd);
  if (st != SFT_OK) return st;
  st = gemm_wgrad(h, 1, 16, (int)ntok, h->ones, 1, 1, h->dD, 16, 0, h->G + h->obd);
  if (st != SFT_OK) return st;
  st = gemm(h, (int)ntok, C, 16, h->dD, 16, 0, 0, h->P + h->oWd, 16, 0, 1, h->dH, C, 0, 1.f, 0.f, nullptr, 1);
  if (st != SFT_OK) return st;
  for (int l = h->L - 1; l >= 0; --l) {
    // h_{l+1} = u + a W2 + b2
    SFS_CUDA(cudaMemcpyAsync(h->dU, h->dH, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm_wgrad(h, 2 * C, C, (int)ntok, h->A[l], 2 * C, 1, h->dH, C, 0, h->G + h->oW2[l]);
    if (st != SFT_OK) return st;
    st = gemm_wgrad(h, 1, C, (int)ntok, h->ones, 1, 1, h->dH, C, 0, h->G + h->ob2[l]);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, 2 * C, C, h->dH, C, 0, 0, h->P + h->oW2[l], C, 0, 1, h->dA, 2 * C, 0, 1.f, 0.f, nullptr, 1);
    if (st != SFT_OK) return st;
    gelu_bwd_kernel<<<grid_for(ntok * 2 * C), 256, 0, h->stream>>>(h->dA, h->Z[l], ntok * 2 * C, h->dZ);
    h->kernels += 1;
    st = gemm_wgrad(h, C, 2 * C, (int)ntok, h->U[l], C, 1, h->dZ, 2 * C, 0, h->G + h->oW1[l]);
    if (st != SFT_OK) return st;
    st = gemm_wgrad(h, 1, 2 * C, (int)ntok, h->ones, 1, 1, h->dZ, 2 * C, 0, h->G + h->ob1[l]);
    if (st != SFT_OK) return st;
    st = gemm(h, (int)ntok, C, 2 * C, h->dZ, 2 * C, 0, 0, h->P + h->oW1[l], 2 * C, 0, 1, h->dU, C, 0, 1.f, 1.f,
              nullptr, 1);
    if (st != SFT_OK) return st;
    // u = h + Gm (w (.) Fm h)
    st = gemm(h, 2 * M, C, WT, h->Gm, 2 * M, 0, 1, h->dU, C, (long long)WT * C, 0, h->dYh, C, (long long)2 * M * C,
              1.f, 0.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
    spectral_bwd_w_kernel<<<grid_for((long long)HT * M * C), 256, 0, h->stream>>>(h->dYh, h->Hh[l], nb, M, C,
                                                                                  h->G + h->ow[l]);
    spectral_bwd_x_kernel<<<grid_for((long long)nb * HT * M * C), 256, 0, h->stream>>>(h->dYh, h->P + h->ow[l], nb,
                                                                                        M, C, h->dHh);
    h->kernels += 2;
    SFS_CUDA(cudaMemcpyAsync(h->dH, h->dU, ntok * C * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    st = gemm(h, WT, C, 2 * M, h->Fm, WT, 0, 1, h->dHh, C, (long long)2 * M * C, 0, h->dH, C, (long long)WT * C, 1.f,
              1.f, nullptr, nb * HT);
    if (st != SFT_OK) return st;
  }
  st = gemm_wgrad(h, KE, C, (int)ntok, h->E, KE, 1, h->dH, C, 0, h->G + h->oWe);
  if (st != SFT_OK) return st;
  st = gemm_wgrad(h, 1, C, (int)ntok, h->ones, 1, 1, h->dH, C, 0, h->G + h->obe);
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
  CR(dalloc(h, &h->ones, ntok));
  fill_kernel<<<grid_for(ntok), 256, 0, h->stream>>>(h->ones, ntok, 1.f);
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
  if (cudaMallocHost(&h->hsums, 2 * nb * sizeof(double)) != cudaSuccess) return bail(fail("pinned alloc failed"));
  if (cudaMallocHost(&h->hlsum, 3 * nb * sizeof(double)) != cudaSuccess) return bail(fail("pinned alloc failed"));
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
  if (h->hsums) cudaFreeHost(h->hsums);
  if (h->hlsum) cudaFreeHost(h->hlsum);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return SFT_OK;
}

int64_t sfs_num_params(sfs_handle h) { return h ? h->np : 0; }

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
  SFS_CUDA(cudaStreamSynchronize(h->stream));
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
    SFS_CUDA(cudaStreamSynchronize(h->stream));
    *loss = host_loss(h, n);
  }
  return SFT_OK;
}

sft_status sfs_rel_l2(sfs_handle h, const float* a, const float* b, int32_t n, double* out) {
  sft_status st = check_batch(h, a, b, n);
  if (st != SFT_OK) return st;
  if (!out) return fail("NULL output", SFT_ERR_ARG);
  sumsq_kernel<<<dim3(kRedBlocks, n), 256, 0, h->stream>>>(a, b, n, h->mpart);
  fold_map_sums<<<n, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->sums);
  h->kernels += 2;
  SFS_CUDA(cudaGetLastError());
  SFS_CUDA(cudaMemcpyAsync(h->hsums, h->sums, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
  for (int i = 0; i < n; ++i) out[i] = std::sqrt(h->hsums[2 * i] / h->hsums[2 * i + 1]);
  return SFT_OK;
}

sft_status sfs_flux(sfs_handle h, const float* maps, int32_t n, double* out) {
  sft_status st = check_batch(h, maps, maps, n);
  if (st != SFT_OK) return st;
  if (!out) return fail("NULL output", SFT_ERR_ARG);
  flux_kernel<<<dim3(kRedBlocks, n), 256, 0, h->stream>>>(maps, h->area, h->mpart);
  fold_map_sums<<<n, 32, 0, h->stream>>>(h->mpart, kRedBlocks, 2, h->sums);
  h->kernels += 2;
  SFS_CUDA(cudaGetLastError());
  SFS_CUDA(cudaMemcpyAsync(out, h->sums, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SFS_CUDA(cudaStreamSynchronize(h->stream));
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
