// sfs_fused.cu -- the surrogate's inference forward pass as one persistent
// kernel (C = 64 channels, 48 latent modes, up to 4 blocks).
//
// A block owns one latent row of one map at a time: 128 tokens x 64
// channels.  All BF16 weights (the latent DFT pair, the embedding, every
// block's channel MLP, the decoder) and the FP32 biases sit in shared memory
// for the whole launch (195 KB for 4 blocks), so HBM sees only the input
// maps, the spectral weights and the output.  Every contraction is a BF16
// tensor-core product with FP32 accumulation (mma.sync m16n8k16), at the
// same rounding points as the unfused path (operands rounded to BF16, sums
// and residuals in FP32):
//   G1  h  = E We + be                     warp w: tokens 16w..16w+15
//   G2  Hh = Fm h                          warp w: channels 8w..8w+7, all 96 modes
//       Yh = w_l,i (.) Hh  (complex, in registers: a thread holds the real
//            and imaginary rows of its modes)
//   G3  u  = h + Gm Yh                     warp w: tokens 16w..
//   G4  z  = u W1 + b1, a = gelu(z)        A operand from G3's registers
//                                          (hardware tanh: see gelu2)
//   G5  h  = u + a W2 + b2                 A operand from G4's registers
//   G6  d  = h Wd + bd  -> unpatched delta rows
// The accumulators of two adjacent 8-column tiles are exactly the A fragment
// of one 16-wide k step, so G3 -> G4 -> G5 -> G6 stay in registers; only G2
// (which mixes all tokens) needs h in shared memory.  Shared layouts: rows of
// 8 or 16 chunks of 16 bytes are XOR-swizzled by (row & 7); others have an
// odd chunk stride; both keep ldmatrix free of bank conflicts.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "sfs_fused.cuh"

namespace sfs_fused {
namespace {

constexpr int H = 256, W = 512, PATCH = 4, HT = 64, C = kChannels, M = kModes;
constexpr float SCALE = 100.0f;
constexpr int kThreads = 256;

// image layout (bytes)
constexpr int FM_OFF = 0;                        // Fm [96][128], 16 chunks / row, swizzled
constexpr int GM_OFF = FM_OFF + 96 * 256;        // Gm [128][96], 13 chunks / row
constexpr int GM_STRIDE = 208;
constexpr int WE_OFF = GM_OFF + 128 * GM_STRIDE;  // We^T [64][48], 7 chunks / row
constexpr int WE_STRIDE = 112;
constexpr int WD_OFF = WE_OFF + 64 * WE_STRIDE;   // Wd^T [16][64], 8 chunks / row, swizzled
constexpr int BIAS_OFF = WD_OFF + 16 * 128;       // FP32 be[64], bd[16], b1[L][128], b2[L][64]
constexpr int E_STRIDE = 112;                     // E [128][48], 7 chunks / row

__host__ __device__ constexpr int bias_floats(int L) { return 64 + 16 + L * (2 * C + C); }
__host__ __device__ constexpr int w1_off(int L) { return (BIAS_OFF + bias_floats(L) * 4 + 127) / 128 * 128; }
__host__ __device__ constexpr int img_bytes(int L) { return w1_off(L) + L * 32768; }  // W1^T, W2^T per block
__host__ __device__ constexpr int hb_off(int L) { return img_bytes(L); }            // h [128][64] BF16, swizzled
__host__ __device__ constexpr int ey_off(int L) { return hb_off(L) + 128 * 128; }   // E, or Yh [96][64] swizzled
__host__ __device__ constexpr int total_smem(int L) { return ey_off(L) + 128 * E_STRIDE; }

// byte offset of 16-byte chunk `chunk` of row `row` in a swizzled array of
// rows of `row_bytes` (a multiple of 128)
__host__ __device__ __forceinline__ int swz(int row, int chunk, int row_bytes) {
  return row * row_bytes + ((chunk ^ (row & 7)) << 4);
}

__device__ __forceinline__ void ldsm4(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void ldsm4t(uint32_t (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

__device__ __forceinline__ void mma(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared.b32 [%0], %1;\n" ::"r"(addr), "r"(v) : "memory");
}

// tanh-form GELU of a pair, 0.5 z (1 + tanh(c z (1 + 0.044715 z^2))), with the
// hardware tanh approximation (tanh.approx.f32, ~2^-11 relative: the result
// is rounded to BF16, 2^-8, right after) and packed f32x2 arithmetic.  The
// training path keeps the accurate tanhf.
__device__ __forceinline__ float tanh_hw(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;\n" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 c = make_float2(0.7978845608028654f, 0.7978845608028654f);
  const float2 k = make_float2(0.044715f, 0.044715f), one = make_float2(1.f, 1.f), half = make_float2(0.5f, 0.5f);
  const float2 z2 = __fmul2_rn(z, z);
  const float2 arg = __fmul2_rn(__fmul2_rn(c, z), __ffma2_rn(k, z2, one));
  const float2 t = make_float2(tanh_hw(arg.x), tanh_hw(arg.y));
  return __fmul2_rn(__fmul2_rn(half, z), __fadd2_rn(one, t));
}

// A fragments (k steps of 16) from accumulators over 2*KS tiles of 8 columns
template <int KS>
__device__ __forceinline__ void acc_to_a(const float (&acc)[2 * KS][4], uint32_t (&a)[KS][4]) {
#pragma unroll
  for (int j = 0; j < KS; ++j) {
    a[j][0] = pack2(acc[2 * j][0], acc[2 * j][1]);
    a[j][1] = pack2(acc[2 * j][2], acc[2 * j][3]);
    a[j][2] = pack2(acc[2 * j + 1][0], acc[2 * j + 1][1]);
    a[j][3] = pack2(acc[2 * j + 1][2], acc[2 * j + 1][3]);
  }
}

struct SpecPtrs {
  const float* w[kMaxBlocks];
};

template <int L>
__global__ void __launch_bounds__(kThreads, 1)
fused_forward_kernel(const unsigned char* __restrict__ img, SpecPtrs ws, const float* __restrict__ x,
                     const float* __restrict__ r, const float* __restrict__ prm, int nrows,
                     float* __restrict__ delta) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, g = lane >> 2, t = lane & 3;
  for (int o = tid * 16; o < img_bytes(L); o += kThreads * 16)
    *reinterpret_cast<uint4*>(smem + o) = *reinterpret_cast<const uint4*>(img + o);
  __syncthreads();
  const uint32_t sb = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  const uint32_t sFm = sb + FM_OFF, sGm = sb + GM_OFF, sWe = sb + WE_OFF, sWd = sb + WD_OFF;
  const uint32_t sW1 = sb + w1_off(L), sHb = sb + hb_off(L), sEY = sb + ey_off(L);
  const float* bias = reinterpret_cast<const float*>(smem + BIAS_OFF);
  const int r16 = 16 * warp;  // this warp's first token (G1, G3..G6)
  // lane -> (row, chunk) of the four 8x8 matrices of an x4 ldmatrix
  const int la = lane & 15, lh = lane >> 4;                                  // A: rows 0..15, chunk +0/+1
  const int lbn = (lane & 7) + ((lane >> 4) << 3), lbk = (lane >> 3) & 1;   // B [n][k]: 2 n tiles x 2 k halves
  const int ltk = ((lane >> 3) & 1) * 8 + (lane & 7), ltn = lane >> 4;      // B [k][n] (trans)

  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int b = row >> 6, i = row & (HT - 1);
    // ---- E: [x patch | r patch | normalised parameters, cos, sin | 0] ----
    {
      const int tok = tid >> 1;
      unsigned char* er = smem + ey_off(L) + tok * E_STRIDE;
      const float inv = 1.0f / SCALE;
      const float* src = (tid & 1) ? r : x;
      uint32_t q[8];
#pragma unroll
      for (int pr = 0; pr < PATCH; ++pr) {
        const float4 v =
            *reinterpret_cast<const float4*>(src + ((long long)b * H + i * PATCH + pr) * W + tok * PATCH);
        q[2 * pr] = pack2(v.x * inv, v.y * inv);
        q[2 * pr + 1] = pack2(v.z * inv, v.w * inv);
      }
      const int c0 = (tid & 1) * 2;
      *reinterpret_cast<uint4*>(er + c0 * 16) = make_uint4(q[0], q[1], q[2], q[3]);
      *reinterpret_cast<uint4*>(er + c0 * 16 + 16) = make_uint4(q[4], q[5], q[6], q[7]);
      if (tid & 1) {
        const float* pp = prm + 5 * b;
        const float n0 = (pp[0] - 13.38f) / 1.338f, n1 = (pp[1] + 2.30f) / 0.230f;
        const float n2 = (pp[2] + 1.62f) / 0.162f, n3 = (pp[3] - 15.0f) / 5.0f;
        const float n4 = (pp[4] - 500.0f) / 250.0f;
        float sn, cs;  // colatitude of the patch row, (i + 1/2) PATCH pi / (H - 1)
        sincospif((i + 0.5f) * PATCH / (H - 1), &sn, &cs);
        *reinterpret_cast<uint4*>(er + 64) =
            make_uint4(pack2(n0, n1), pack2(n2, n3), pack2(n4, cs), pack2(sn, 0.f));
        *reinterpret_cast<uint4*>(er + 80) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    __syncthreads();
    // ---- G1: h = E We + be ----
    float hres[8][4];
#pragma unroll
    for (int n = 0; n < 8; ++n)
#pragma unroll
      for (int q = 0; q < 4; ++q) hres[n][q] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 3; ++ks) {
      uint32_t a[4];
      ldsm4(a, sEY + (r16 + la) * E_STRIDE + ((2 * ks + lh) << 4));
#pragma unroll
      for (int np = 0; np < 4; ++np) {
        uint32_t bq[4];
        ldsm4(bq, sWe + (16 * np + lbn) * WE_STRIDE + ((2 * ks + lbk) << 4));
        mma(hres[2 * np], a, bq[0], bq[1]);
        mma(hres[2 * np + 1], a, bq[2], bq[3]);
      }
    }
#pragma unroll
    for (int n = 0; n < 8; ++n) {
      const int c = 8 * n + 2 * t;
      hres[n][0] += bias[c];
      hres[n][1] += bias[c + 1];
      hres[n][2] += bias[c];
      hres[n][3] += bias[c + 1];
      sts32(sHb + swz(r16 + g, n, 128) + 4 * t, pack2(hres[n][0], hres[n][1]));
      sts32(sHb + swz(r16 + g + 8, n, 128) + 4 * t, pack2(hres[n][2], hres[n][3]));
    }
    __syncthreads();
#pragma unroll 1
    for (int l = 0; l < L; ++l) {
      // ---- G2: Hh = Fm h (this warp: channels 8w..8w+7, modes 0..95) ----
      float hh[6][4];
#pragma unroll
      for (int m = 0; m < 6; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q) hh[m][q] = 0.f;
#pragma unroll
      for (int kp = 0; kp < 4; ++kp) {
        uint32_t bb[4];  // B fragments of k steps 2kp (bb[0..1]) and 2kp+1 (bb[2..3])
        ldsm4t(bb, sHb + swz(32 * kp + lane, warp, 128));
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          const int ks = 2 * kp + kk;
#pragma unroll
          for (int m = 0; m < 6; ++m) {
            uint32_t a[4];
            ldsm4(a, sFm + swz(16 * m + la, 2 * ks + lh, 256));
            mma(hh[m], a, bb[2 * kk], bb[2 * kk + 1]);
          }
        }
      }
      // Yh = w (.) Hh; a thread holds modes 16m+g (+8) real (m < 3) and imaginary (m + 3)
      {
        const float* wl = ws.w[l] + (long long)i * M * C * 2;
        const int c = 8 * warp + 2 * t;
#pragma unroll
        for (int m = 0; m < 3; ++m)
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            const int k = 16 * m + g + 8 * hf;
            const float2 w0 = *reinterpret_cast<const float2*>(wl + ((long long)k * C + c) * 2);
            const float2 w1 = *reinterpret_cast<const float2*>(wl + ((long long)k * C + c + 1) * 2);
            const float hr0 = hh[m][2 * hf], hr1 = hh[m][2 * hf + 1];
            const float hi0 = hh[m + 3][2 * hf], hi1 = hh[m + 3][2 * hf + 1];
            sts32(sEY + swz(k, warp, 128) + 4 * t, pack2(w0.x * hr0 - w0.y * hi0, w1.x * hr1 - w1.y * hi1));
            sts32(sEY + swz(M + k, warp, 128) + 4 * t, pack2(w0.x * hi0 + w0.y * hr0, w1.x * hi1 + w1.y * hr1));
          }
      }
      __syncthreads();
      // ---- G3: u = h + Gm Yh (accumulated onto h) ----
#pragma unroll
      for (int ks = 0; ks < 6; ++ks) {
        uint32_t a[4];
        ldsm4(a, sGm + (r16 + la) * GM_STRIDE + ((2 * ks + lh) << 4));
#pragma unroll
        for (int np = 0; np < 4; ++np) {
          uint32_t bq[4];
          ldsm4t(bq, sEY + swz(16 * ks + ltk, 2 * np + ltn, 128));
          mma(hres[2 * np], a, bq[0], bq[1]);
          mma(hres[2 * np + 1], a, bq[2], bq[3]);
        }
      }
      // ---- G4: z = u W1 + b1, a = gelu(z) ----
      uint32_t za[8][4];
      {
        uint32_t ua[4][4];
        acc_to_a<4>(hres, ua);
        float z[16][4];
#pragma unroll
        for (int n = 0; n < 16; ++n)
#pragma unroll
          for (int q = 0; q < 4; ++q) z[n][q] = 0.f;
        const uint32_t w1 = sW1 + l * 32768;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
#pragma unroll
          for (int np = 0; np < 8; ++np) {
            uint32_t bq[4];
            ldsm4(bq, w1 + swz(16 * np + lbn, 2 * ks + lbk, 128));
            mma(z[2 * np], ua[ks], bq[0], bq[1]);
            mma(z[2 * np + 1], ua[ks], bq[2], bq[3]);
          }
        const float* b1 = bias + 80 + l * 2 * C;
#pragma unroll
        for (int n = 0; n < 16; ++n) {
          const float2 bb = *reinterpret_cast<const float2*>(b1 + 8 * n + 2 * t);
          const float2 lo = gelu2(__fadd2_rn(make_float2(z[n][0], z[n][1]), bb));
          const float2 hi = gelu2(__fadd2_rn(make_float2(z[n][2], z[n][3]), bb));
          z[n][0] = lo.x;
          z[n][1] = lo.y;
          z[n][2] = hi.x;
          z[n][3] = hi.y;
        }
        acc_to_a<8>(z, za);
      }
      // ---- G5: h = u + a W2 + b2 (accumulated onto u) ----
      {
        const uint32_t w2 = sW1 + l * 32768 + 16384;
#pragma unroll
        for (int ks = 0; ks < 8; ++ks)
#pragma unroll
          for (int np = 0; np < 4; ++np) {
            uint32_t bq[4];
            ldsm4(bq, w2 + swz(16 * np + lbn, 2 * ks + lbk, 256));
            mma(hres[2 * np], za[ks], bq[0], bq[1]);
            mma(hres[2 * np + 1], za[ks], bq[2], bq[3]);
          }
        const float* b2 = bias + 80 + L * 2 * C + l * C;
#pragma unroll
        for (int n = 0; n < 8; ++n) {
          const int c = 8 * n + 2 * t;
          hres[n][0] += b2[c];
          hres[n][1] += b2[c + 1];
          hres[n][2] += b2[c];
          hres[n][3] += b2[c + 1];
          if (l + 1 < L) {
            sts32(sHb + swz(r16 + g, n, 128) + 4 * t, pack2(hres[n][0], hres[n][1]));
            sts32(sHb + swz(r16 + g + 8, n, 128) + 4 * t, pack2(hres[n][2], hres[n][3]));
          }
        }
      }
      __syncthreads();
    }
    // ---- G6: d = h Wd + bd, written as the unpatched delta rows ----
    {
      uint32_t ha[4][4];
      acc_to_a<4>(hres, ha);
      float d[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        uint32_t bq[4];
        ldsm4(bq, sWd + swz(lbn, 2 * ks + lbk, 128));
        mma(d[0], ha[ks], bq[0], bq[1]);
        mma(d[1], ha[ks], bq[2], bq[3]);
      }
      const float* bd = bias + 64;
#pragma unroll
      for (int n = 0; n < 2; ++n) {
        const int o = 8 * n + 2 * t, pr = o >> 2, pc = o & 3;
        float* dr = delta + ((long long)b * H + i * PATCH + pr) * W + pc;
        *reinterpret_cast<float2*>(dr + (r16 + g) * PATCH) = make_float2(d[n][0] + bd[o], d[n][1] + bd[o + 1]);
        *reinterpret_cast<float2*>(dr + (r16 + g + 8) * PATCH) = make_float2(d[n][2] + bd[o], d[n][3] + bd[o + 1]);
      }
    }
  }
}

// One thread per destination element of the image.
__global__ void build_image_kernel(const float* __restrict__ P, ParamOffsets o, int L,
                                   const float* __restrict__ Fm, const float* __restrict__ Gm,
                                   unsigned char* __restrict__ img) {
  const int n_fm = 96 * 128, n_gm = 128 * 96, n_we = 64 * 48, n_wd = 16 * 64, n_b = bias_floats(L);
  const int n_w = 2 * C * C;  // per matrix
  const long long total = (long long)n_fm + n_gm + n_we + n_wd + n_b + 2LL * L * n_w;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    long long q = e;
    auto put = [&](int byte, float v) { *reinterpret_cast<__nv_bfloat16*>(img + byte) = __float2bfloat16_rn(v); };
    if (q < n_fm) {
      const int rr = (int)q / 128, k = (int)q % 128;
      put(FM_OFF + swz(rr, k >> 3, 256) + (k & 7) * 2, Fm[q]);
      continue;
    }
    q -= n_fm;
    if (q < n_gm) {
      const int rr = (int)q / 96, k = (int)q % 96;
      put(GM_OFF + rr * GM_STRIDE + k * 2, Gm[q]);
      continue;
    }
    q -= n_gm;
    if (q < n_we) {  // We^T[n][k] = We[k][n]
      const int n = (int)q / 48, k = (int)q % 48;
      put(WE_OFF + n * WE_STRIDE + k * 2, P[o.We + (long long)k * C + n]);
      continue;
    }
    q -= n_we;
    if (q < n_wd) {  // Wd^T[out][c] = Wd[c][out]
      const int out = (int)q / 64, c = (int)q % 64;
      put(WD_OFF + swz(out, c >> 3, 128) + (c & 7) * 2, P[o.Wd + (long long)c * 16 + out]);
      continue;
    }
    q -= n_wd;
    if (q < n_b) {
      float v;
      if (q < 64) v = P[o.be + q];
      else if (q < 80) v = P[o.bd + (q - 64)];
      else if (q < 80 + L * 2 * C) v = P[o.b1[(q - 80) / (2 * C)] + (q - 80) % (2 * C)];
      else v = P[o.b2[(q - 80 - L * 2 * C) / C] + (q - 80 - L * 2 * C) % C];
      reinterpret_cast<float*>(img + BIAS_OFF)[q] = v;
      continue;
    }
    q -= n_b;
    const int l = (int)(q / (2 * n_w));
    q -= (long long)l * 2 * n_w;
    const int base = w1_off(L) + l * 32768;
    if (q < n_w) {  // W1^T[j][c] = W1[c][j], j < 128, c < 64
      const int j = (int)q / C, c = (int)q % C;
      put(base + swz(j, c >> 3, 128) + (c & 7) * 2, P[o.W1[l] + (long long)c * 2 * C + j]);
    } else {  // W2^T[c][j] = W2[j][c]
      q -= n_w;
      const int c = (int)q / (2 * C), j = (int)q % (2 * C);
      put(base + 16384 + swz(c, j >> 3, 256) + (j & 7) * 2, P[o.W2[l] + (long long)j * C + c]);
    }
  }
}

template <int L>
cudaError_t launch(const unsigned char* img, const float* P, const ParamOffsets& o, const float* x, const float* r,
                   const float* p, int nb, float* delta, int n_sm, cudaStream_t st) {
  SpecPtrs ws{};
  for (int l = 0; l < L; ++l) ws.w[l] = P + o.w[l];
  const int nrows = nb * HT;
  const int grid = nrows < n_sm ? nrows : n_sm;
  fused_forward_kernel<L><<<grid, kThreads, total_smem(L), st>>>(img, ws, x, r, p, nrows, delta);
  return cudaGetLastError();
}

template <int L>
cudaError_t prepare_l() {
  return cudaFuncSetAttribute(fused_forward_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, total_smem(L));
}

}  // namespace

size_t image_bytes(int L) { return (size_t)img_bytes(L); }
size_t smem_bytes(int L) { return (size_t)total_smem(L); }

cudaError_t prepare(int L) {
  switch (L) {
    case 1: return prepare_l<1>();
    case 2: return prepare_l<2>();
    case 3: return prepare_l<3>();
    case 4: return prepare_l<4>();
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t build_image(const float* P, const ParamOffsets& o, int L, const float* Fm, const float* Gm,
                        unsigned char* img, cudaStream_t st) {
  if (L < 1 || L > kMaxBlocks) return cudaErrorInvalidValue;
  build_image_kernel<<<152 * 4, 256, 0, st>>>(P, o, L, Fm, Gm, img);
  return cudaGetLastError();
}

cudaError_t forward(const unsigned char* img, int L, const float* P, const ParamOffsets& o, const float* x,
                    const float* r, const float* p, int nb, float* delta, int n_sm, cudaStream_t st) {
  switch (L) {
    case 1: return launch<1>(img, P, o, x, r, p, nb, delta, n_sm, st);
    case 2: return launch<2>(img, P, o, x, r, p, nb, delta, n_sm, st);
    case 3: return launch<3>(img, P, o, x, r, p, nb, delta, n_sm, st);
    case 4: return launch<4>(img, P, o, x, r, p, nb, delta, n_sm, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace sfs_fused
