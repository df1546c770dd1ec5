// sft_kernels.cu -- sm_103a kernels of the SFT step.
//
//  rkl2_stage_kernel  one RKL2 stage (Sec. 3.7.2) of the 5-point diffusion
//                     operator of Eq. (diffusion_op) with constant nu and the
//                     polar caps of App. A, in increment form (see below).
//  adv_stage_kernel   one SSPRK / FE stage (Sec. 3.6.2) of the conservative
//                     advection operator of Sec. 3.6.1 with WENO3-CS(h)
//                     (App. B) or UW face fluxes and the App. A caps.
//  reduce/fold/apply  FP64 reductions for the analysis quantities (Sec. 2.6),
//                     the assimilation balance (Sec. 2.3) and map balancing.
//
// All stage kernels are HBM-streaming stencils: one 16-byte vector per
// thread per array, phi neighbours through warp shuffles (global loads only
// at warp edges, the periodic seam and the ragged last tile), theta
// neighbours as vector loads of the adjacent rows (served by L2 when the
// adjacent tile ran just before).
#include <math.h>

#include "sft_device.cuh"

namespace sft {

#ifdef SFT_DEBUG
namespace {
__device__ unsigned long long g_dbg_first;  // (site << 48) | (value mod 2^48) of the first failed check
__device__ unsigned int g_dbg_count;        // failed checks

__global__ void debug_probe_kernel(int site, int64_t v, int64_t lo, int64_t hi) {
  (void)dbg_check(site, v, lo, hi);
}
}  // namespace

__device__ void dbg_record(int site, int64_t v) {
  const unsigned long long w =
      ((unsigned long long)(site & 0xffff) << 48) | ((unsigned long long)v & ((1ull << 48) - 1));
  atomicCAS(&g_dbg_first, 0ull, w);
  atomicAdd(&g_dbg_count, 1u);
}

cudaError_t debug_read(uint64_t* first, uint32_t* count, bool reset) {
  cudaError_t e = cudaDeviceSynchronize();  // side streams included
  unsigned long long f = 0;
  unsigned int c = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, g_dbg_first, sizeof(f));
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&c, g_dbg_count, sizeof(c));
  if (e != cudaSuccess) return e;
  if (first) *first = f;
  if (count) *count = c;
  if (reset) {
    f = 0;
    c = 0;
    e = cudaMemcpyToSymbol(g_dbg_first, &f, sizeof(f));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_dbg_count, &c, sizeof(c));
  }
  return e;
}

cudaError_t launch_debug_probe(int site, int64_t v, int64_t lo, int64_t hi, cudaStream_t st) {
  debug_probe_kernel<<<1, 1, 0, st>>>(site, v, lo, hi);
  return cudaGetLastError();
}
#else
cudaError_t debug_read(uint64_t*, uint32_t*, bool) { return cudaErrorNotSupported; }
cudaError_t launch_debug_probe(int, int64_t, int64_t, int64_t, cudaStream_t) { return cudaErrorNotSupported; }
#endif

namespace {

template <typename T> struct Vec;
template <> struct Vec<float> {
  static constexpr int N = 4;
  __device__ __forceinline__ static void ldg(const float* p, float (&c)[4]) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
  }
  __device__ __forceinline__ static void ld(const float* p, float (&c)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
  }
  __device__ __forceinline__ static void st(float* p, const float (&c)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(c[0], c[1], c[2], c[3]);
  }
};
template <> struct Vec<double> {
  static constexpr int N = 2;
  __device__ __forceinline__ static void ldg(const double* p, double (&c)[2]) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    c[0] = v.x; c[1] = v.y;
  }
  __device__ __forceinline__ static void ld(const double* p, double (&c)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    c[0] = v.x; c[1] = v.y;
  }
  __device__ __forceinline__ static void st(double* p, const double (&c)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(c[0], c[1]);
  }
};

// e[H + i] = row value at column kc + i (periodic), for i = -H .. N+H-1.
// Every lane of the warp must call this (warp shuffles); lanes with kc >= np
// skip their global loads and get undefined e.
template <typename T, int N, int H>
__device__ __forceinline__ void row_ext(const T* __restrict__ row, int kc, int np, int lane,
                                        const T (&c)[N], T (&e)[N + 2 * H]) {
#pragma unroll
  for (int i = 0; i < N; ++i) e[H + i] = c[i];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    e[H - 1 - m] = __shfl_up_sync(0xffffffffu, c[N - 1 - m], 1);
    e[H + N + m] = __shfl_down_sync(0xffffffffu, c[m], 1);
  }
  if (kc >= np) return;
  if (lane == 0 || kc == 0) {
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const int k = kc - 1 - m;
      e[H - 1 - m] = row[k < 0 ? k + np : k];
    }
  }
  if (lane == 31 || kc + N >= np) {
#pragma unroll
    for (int m = 0; m < H; ++m) {
      const int k = kc + N + m;
      e[H + N + m] = row[k >= np ? k - np : k];
    }
  }
  if (kc + N > np) {  // ragged last vector: columns >= np hold the wrapped values
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (kc + i >= np) e[H + i] = row[kc + i - np];
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the block, result returned to every thread.  Contains barriers.
__device__ double block_sum(double v, double* sm) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  double t = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) t += sm[i];  // fixed order: deterministic
  return t;
}

// UW/CD flux at a face (Sec. 3.6.1): v/2 [(1-uw) B_hi + (1+uw) B_lo],
// uw = alpha_uw sign(v), sign(0) = +1.
template <typename T>
__device__ __forceinline__ T uw_flux(T v, T blo, T bhi, T auw) {
  const T uw = v >= T(0) ? auw : -auw;
  return v * T(0.5) * ((T(1) - uw) * bhi + (T(1) + uw) * blo);
}

// The one division of a WENO half-flux: FP32 takes the hardware-approximate
// quotient (__fdividef, a few ulp: far inside the FP32 bar of 1e-5 max|Br|),
// FP64 the IEEE quotient.
__device__ __forceinline__ float weno_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double weno_div(double a, double b) { return a / b; }

// WENO3-CS(h) face flux (App. B) on a uniform grid, from LM_{i-2}, LM_{i-1},
// LM_i and LP_{i-1}, LP_i, LP_{i+1}.  Weight algebra is written as
// w0/(w0+w1) = 1 / (1 + 2 ((eps+b0)/(eps+b1))^2) with linear weights 1/3, 2/3.
template <typename T>
__device__ __forceinline__ T weno_half(T p0, T p1, T b0, T b1, T eps) {
  const T q0 = eps + b0, q1 = eps + b1;
  const T a0 = q1 * q1;            // (1/3)/q0^2 scaled by 3 q0^2 q1^2
  const T a1 = T(2) * q0 * q0;     // (2/3)/q1^2 scaled the same way
  return weno_div(a0 * p0 + a1 * p1, a0 + a1);
}

// The two halves of the split face flux: LM (from LM_{i-2}, LM_{i-1}, LM_i)
// and LP (from LP_{i-1}, LP_i, LP_{i+1}).
template <typename T>
__device__ __forceinline__ T weno_lm(T lmm2, T lmm1, T lm0, T eps) {
  const T dm0 = lmm1 - lmm2, dm1 = lm0 - lmm1;
  return weno_half(T(1.5) * lmm1 - T(0.5) * lmm2, T(0.5) * (lmm1 + lm0), dm0 * dm0, dm1 * dm1, eps);
}
template <typename T>
__device__ __forceinline__ T weno_lp(T lpm1, T lp0, T lpp1, T eps) {
  const T dp0 = lpp1 - lp0, dp1 = lp0 - lpm1;
  return weno_half(T(1.5) * lp0 - T(0.5) * lpp1, T(0.5) * (lp0 + lpm1), dp0 * dp0, dp1 * dp1, eps);
}

template <typename T>
__device__ __forceinline__ T weno_flux(T lmm2, T lmm1, T lm0, T lpm1, T lp0, T lpp1, T eps) {
  return weno_lm(lmm2, lmm1, lm0, eps) + weno_lp(lpm1, lp0, lpp1, eps);
}

}  // namespace

// ---------------------------------------------------------------------------
// RKL2 stage, increment form.
//
// The RKL2 stages Y_j = mu_j Y_{j-1} + nu_j Y_{j-2} + (1-mu_j-nu_j) Y_0
//   + mu~_j dt L(Y_{j-1}) + gamma~_j dt L(Y_0)   (Meyer, Balsara & Aslam 2014)
// are carried as increments delta_j = Y_j - Y_0 (L is linear):
//   G = dt L(Y_0),  delta_1 = mu~_1 G,
//   delta_j = mu_j delta_{j-1} + nu_j delta_{j-2} + mu~_j dt L(delta_{j-1})
//             + (mu~_j + gamma~_j) G,
//   Y_s = Y_0 + delta_s   (written to the state by the last stage).
// Identical in exact arithmetic; in FP32 the rounding is relative to the
// increment, not to |B|.  Per stage HBM traffic: read delta_{j-1},
// delta_{j-2}, G; write delta_j (over delta_{j-2}) = 16 B per cell (FP32).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
rkl2_stage_kernel(const Tile* __restrict__ tiles, const RealDesc* __restrict__ rd,
                  const StepParam* __restrict__ sp, const RowGeo<T>* __restrict__ geo,
                  const ShapeConst* __restrict__ shc, const Coef<T>* __restrict__ coef,
                  T* __restrict__ B, T* __restrict__ G, T* __restrict__ D0, T* __restrict__ D1,
                  int stage, int allow_final, int* __restrict__ status) {
  constexpr int N = Vec<T>::N;
  __shared__ double sm[kThreads / 32];
  const Tile tl = tiles[blockIdx.x];
  const int kind = tl.kind & 3, lx = tl.kind >> 8;  // lx = log2(threads per tile row)
  const RealDesc d = rd[tl.r];
  const StepParam p = sp[tl.r];
  if (stage > p.s) return;
  const bool first = stage == 1;
  const bool last = stage == p.s && allow_final;
  const Coef<T> cf = coef[p.coef + stage];
  const T nudt = T(p.nudt);
  T* Dout = ((stage & 1) ? D1 : D0) + d.woff;          // delta_j (over delta_{j-2})
  const T* Din = ((stage & 1) ? D0 : D1) + d.woff;     // delta_{j-1}
  T* Gw = G + d.woff;
  T* Bs = B + d.off;
  const T* Y = first ? Bs : Din;
  const int pitch = d.pitch, np = d.np;

  if (kind != 0) {
    // App. A cap: div(nu grad B) = sin(dth/2) dph sum_k nu (Y_adj,k - Y_p)/dth / cap
    const int jp = kind == 1 ? 0 : d.nt - 1;
    const int ja = kind == 1 ? 1 : d.nt - 2;
    const T* ya = Y + (int64_t)ja * pitch;
    const double yp = double(Y[(int64_t)jp * pitch]);
    double acc = 0.0;
    for (int k = threadIdx.x; k < np; k += blockDim.x) acc += double(ya[k]) - yp;
    const int64_t po = (int64_t)jp * pitch;
    // pointwise pole operands, read before the barrier inside block_sum
    double gp = 0.0, d2 = 0.0, b0 = 0.0;
    if (!first) {
      gp = double(Gw[po]);
      if (stage > 2) d2 = double(Dout[po]);
      if (last) b0 = double(Bs[po]);
    }
    const double Lp = shc[d.shape].pole_diff * p.cap_nu * block_sum(acc, sm);
    if (first) {
      const T g = T(double(nudt) * Lp);
      const T o = cf.mut * g;
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        Gw[po + k] = g;
        Dout[po + k] = o;
      }
    } else {
      const double o = double(cf.mu) * yp + double(cf.nu) * d2 +
                       double(cf.mut) * double(nudt) * Lp + double(cf.gsum) * gp;
      if (last) {
        const T v = T(b0 + o);
        if (threadIdx.x == 0 && !isfinite(double(v))) atomicOr(status, 1);
        for (int k = threadIdx.x; k < np; k += blockDim.x) Bs[po + k] = v;
      } else {
        const T v = T(o);
        for (int k = threadIdx.x; k < np; k += blockDim.x) Dout[po + k] = v;
      }
    }
    return;
  }

  const int ty = threadIdx.x >> lx, tx = threadIdx.x & ((1 << lx) - 1), lane = threadIdx.x & 31;
  int j = tl.j0 + ty;
  if (j > d.nt - 2) return;  // a warp lies within one row: uniform exit
  SFT_DCHECK(DBG_STAGE_ROW, j, 1, d.nt - 2);
  int kc = tl.k0 + tx * N;
  if (kc < np) SFT_DCHECK(DBG_STAGE_COL, kc, 0, min(np - 1, pitch - N));
  const int64_t ro = (int64_t)j * pitch;
  T c[N], up[N], dn[N];
  if (kc < np) {
    Vec<T>::ldg(Y + ro + kc, c);
    Vec<T>::ldg(Y + ro - pitch + kc, up);
    Vec<T>::ldg(Y + ro + pitch + kc, dn);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) c[i] = up[i] = dn[i] = T(0);
  }
  T e[N + 2];
  row_ext<T, N, 1>(Y + ro, kc, np, lane, c, e);
  if (kc >= np) return;
  const RowGeo<T> g = geo[d.geo + j];
  T L[N];
#pragma unroll
  for (int i = 0; i < N; ++i)
    L[i] = g.cN * (up[i] - c[i]) + g.cS * (dn[i] - c[i]) + g.cE * ((e[i] - c[i]) + (e[i + 2] - c[i]));
  T o[N];
  if (first) {
    T gv[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      gv[i] = nudt * L[i];
      o[i] = cf.mut * gv[i];
    }
    Vec<T>::st(Gw + ro + kc, gv);
    Vec<T>::st(Dout + ro + kc, o);
    return;
  }
  T gv[N], d2[N];
  Vec<T>::ldg(Gw + ro + kc, gv);
  if (stage > 2) {
    Vec<T>::ld(Dout + ro + kc, d2);
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) d2[i] = T(0);
  }
  const T mutdt = cf.mut * nudt;
#pragma unroll
  for (int i = 0; i < N; ++i) o[i] = cf.mu * c[i] + cf.nu * d2[i] + mutdt * L[i] + cf.gsum * gv[i];
  if (last) {
    T b[N];
    Vec<T>::ld(Bs + ro + kc, b);
    bool bad = false;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      b[i] += o[i];
      bad |= (kc + i < np) && !isfinite(double(b[i]));
    }
    Vec<T>::st(Bs + ro + kc, b);
    if (bad) atomicOr(status, 1);
  } else {
    Vec<T>::st(Dout + ro + kc, o);
  }
}

// Face fluxes of one advection stage.  ATT: Eq. (flow_attenuation) -- every
// flux term v B_i carries the cell's factor a_i = 1 - tanh(|B_i| / B_0) (the
// upwind flux and the advective part of the LLF split); the dissipative
// alpha B term keeps the unattenuated bound.
//
// A realization's advection constants in the state's type, converted once
// per thread (FP64 conversions run on GB300's narrow FP64 pipe).
template <typename T> struct AdvConst {
  T ib0, eps_p, eps_t, auw;
  bool weno, att;
  __device__ explicit AdvConst(const StepParam& p)
      : ib0(T(p.inv_b0)), eps_p(T(p.eps_p)), eps_t(T(p.eps_t)), auw(T(p.alpha_uw)),
        weno(p.weno != 0), att(p.inv_b0 != 0.0) {}
};

// phi faces k-1/2 of a thread's N points, k = kc .. kc+N, from the row's
// values e (columns kc-2 .. kc+N+1) and v_phi of the row.
template <typename T, int N, bool ATT>
__device__ __forceinline__ void phi_faces(const AdvConst<T>& q, T v, const T (&e)[N + 4], T (&F)[N + 1]) {
  const T ib0 = q.ib0, auw = q.auw;
  auto att = [&](T x) -> T { return ATT ? T(1) - tanh(fabs(x) * ib0) : T(1); };
  if (q.weno) {
    const T eps = q.eps_p;
    const T av = fabs(v);
    if (ATT) {
      T lm[N + 4], lp[N + 4];
#pragma unroll
      for (int i = 0; i < N + 4; ++i) {
        const T vab = v * att(e[i]) * e[i];
        lm[i] = T(0.5) * (vab + av * e[i]);
        lp[i] = T(0.5) * (vab - av * e[i]);
      }
#pragma unroll
      for (int i = 0; i <= N; ++i) F[i] = weno_flux(lm[i], lm[i + 1], lm[i + 2], lp[i + 1], lp[i + 2], lp[i + 3], eps);
    } else if (v >= T(0)) {
      // v_phi is one value per row, so one half of the LLF split vanishes:
      // hm = (v - |v|)/2 = 0 and the LP half-fluxes are zeros (the face flux
      // is the LM half alone, up to the sign of a zero)
      const T hp = T(0.5) * (v + av);
#pragma unroll
      for (int i = 0; i <= N; ++i) F[i] = weno_lm(hp * e[i], hp * e[i + 1], hp * e[i + 2], eps);
    } else {
      const T hm = T(0.5) * (v - av);  // hp = 0: the LP half alone
#pragma unroll
      for (int i = 0; i <= N; ++i) F[i] = weno_lp(hm * e[i + 1], hm * e[i + 2], hm * e[i + 3], eps);
    }
  } else {
#pragma unroll
    for (int i = 0; i <= N; ++i)
      F[i] = ATT ? uw_flux(v, att(e[i + 1]) * e[i + 1], att(e[i + 2]) * e[i + 2], auw)
                 : uw_flux(v, e[i + 1], e[i + 2], auw);
  }
}

// theta face f+1/2 of a thread's N columns from rows f-1 .. f+2 (values R,
// flow rows fl, clamped to the interior): WENO3-CS(h) with the LLF split (LM
// uses v at a cell's lower face, LP at its upper) when `weno`, else UW with
// vface, v_theta at the face (taken from an unclamped row by the caller).
template <typename T, int N, bool ATT>
__device__ __forceinline__ void theta_face(const AdvConst<T>& q, const RowFlow<T> (&fl)[4], const T (&R)[4][N],
                                           bool weno, T vface, T (&F)[N]) {
  const T ib0 = q.ib0, auw = q.auw;
  auto att = [&](T x) -> T { return ATT ? T(1) - tanh(fabs(x) * ib0) : T(1); };
  auto LM = [&](int m, T b) -> T {
    return ATT ? T(0.5) * (fl[m].vdn * att(b) * b + fl[m].alpha * b) : T(0.5) * b * (fl[m].vdn + fl[m].alpha);
  };
  auto LP = [&](int m, T b) -> T {
    return ATT ? T(0.5) * (fl[m].vup * att(b) * b - fl[m].alpha * b) : T(0.5) * b * (fl[m].vup - fl[m].alpha);
  };
  const T eps = q.eps_t;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    if (weno)
      F[i] = weno_flux(LM(0, R[0][i]), LM(1, R[1][i]), LM(2, R[2][i]), LP(1, R[1][i]), LP(2, R[2][i]),
                       LP(3, R[3][i]), eps);
    else
      F[i] = ATT ? uw_flux(vface, att(R[1][i]) * R[1][i], att(R[2][i]) * R[2][i], auw)
                 : uw_flux(vface, R[1][i], R[2][i], auw);
  }
}

// ---------------------------------------------------------------------------
// Advection stage: out = a fn + b fin - c dt F_A(fin).
// F_A(B)_{j,k} = (sin th_{j+1/2} F_{j+1/2} - sin th_{j-1/2} F_{j-1/2}) / (sin th_j dth)
//              + (F_{k+1/2} - F_{k-1/2}) / (sin th_j dph)           (Sec. 3.6.1)
// theta faces f <= 1 and f >= nt-3 (the cap faces and the other face of each
// pole-adjacent cell) use UW; the rest WENO3-CS(h) (or all UW).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
adv_stage_kernel(const Tile* __restrict__ tiles, const RealDesc* __restrict__ rd,
                 const StepParam* __restrict__ sp, const RowGeo<T>* __restrict__ geo,
                 const RowFlow<T>* __restrict__ flow, const ShapeConst* __restrict__ shc,
                 T* __restrict__ state, T* __restrict__ w0, T* __restrict__ w1, AdvStage<T> s) {
  constexpr int N = Vec<T>::N;
  __shared__ double sm[kThreads / 32];
  (void)w0;
  (void)w1;
  const Tile tl = tiles[blockIdx.x];
  const int kind = tl.kind & 3, lx = tl.kind >> 8;
  const RealDesc d = rd[tl.r];
  const StepParam p = sp[tl.r];
  if (p.dt == 0.0 || p.adv == 0) return;
  const T* fin = s.fin + (s.fin_work ? d.woff : d.off);
  const T* fn = s.fn ? s.fn + (s.fn_work ? d.woff : d.off) : nullptr;
  T* out = s.out + (s.out_work ? d.woff : d.off);
  const int pitch = d.pitch, np = d.np, nt = d.nt;
  const T cdt = s.c * T(p.dt_adv);
  const T auw = T(p.alpha_uw);

  if (kind != 0) {
    const bool north = kind == 1;
    const int jp = north ? 0 : nt - 1;
    const int ja = north ? 1 : nt - 2;
    const int64_t po = (int64_t)jp * pitch;
    const T* ba = fin + (int64_t)ja * pitch;
    const T bp = fin[po];
    const T v = north ? flow[d.flow + 1].vdn : flow[d.flow + nt - 2].vup;
    double acc = 0.0;
    if (s.c != T(0)) {
      const T ib0 = T(p.inv_b0);
      const T ap = p.inv_b0 != 0.0 ? (T(1) - tanh(fabs(bp) * ib0)) * bp : bp;  // attenuated pole flux term
      for (int k = threadIdx.x; k < np; k += blockDim.x) {
        const T bk = p.inv_b0 != 0.0 ? (T(1) - tanh(fabs(ba[k]) * ib0)) * ba[k] : ba[k];
        acc += double(north ? uw_flux(v, ap, bk, auw) : uw_flux(v, bk, ap, auw));
      }
    }
    const double fnp = fn ? double(fn[po]) : 0.0;  // read before the barrier
    const double div = (north ? 1.0 : -1.0) * shc[d.shape].pole_adv * block_sum(acc, sm);
    const T o = T(double(s.a) * fnp + double(s.b) * double(bp) - double(s.c) * p.dt_adv * div);
    for (int k = threadIdx.x; k < np; k += blockDim.x) out[po + k] = o;
    return;
  }

  // interior: thread (ty, tx) marches rows jb .. jb+kAdvRun-1 (< nt-1) over
  // its N columns; the theta face between two rows is computed once, as the
  // upper face of the first and carried as the lower face of the second
  const int ty = threadIdx.x >> lx, tx = threadIdx.x & ((1 << lx) - 1), lane = threadIdx.x & 31;
  int jb = tl.j0 + ty * kAdvRun;
  if (jb > nt - 2) return;  // a warp lies within one row group: uniform exit
  SFT_DCHECK(DBG_ADV_ROW, jb, 1, nt - 2);
  const int je = min(jb + kAdvRun, nt - 1);
  int kc = tl.k0 + tx * N;
  if (kc < np) SFT_DCHECK(DBG_ADV_COL, kc, 0, min(np - 1, pitch - N));
  const bool act = kc < np;
  const AdvConst<T> q(p);
  const bool weno = q.weno;
  // five-row windows: values of rows j-2 .. j+2 (clamped to the grid) and
  // flow rows (clamped to the interior)
  T R[5][N];
  RowFlow<T> fl[5];
  auto load_row = [&](int m, int jj) {
    const int jr = jj < 0 ? 0 : (jj > nt - 1 ? nt - 1 : jj);
    if (act) {
      Vec<T>::ldg(fin + (int64_t)jr * pitch + kc, R[m]);
    } else {
#pragma unroll
      for (int i = 0; i < N; ++i) R[m][i] = T(0);
    }
    const int jf = jj < 1 ? 1 : (jj > nt - 2 ? nt - 2 : jj);
    fl[m] = flow[d.flow + jf];
  };
#pragma unroll
  for (int m = 0; m < 4; ++m) load_row(m, jb - 2 + m);
  T Fdn[N];
  if (s.c != T(0) && act) {
    const RowFlow<T> f4[4] = {fl[0], fl[1], fl[2], fl[3]};
    T R4[4][N];
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int i = 0; i < N; ++i) R4[m][i] = R[m][i];
    const bool wdn = weno && (jb - 1 >= 2) && (jb - 1 <= nt - 4);
    // the lower face of row jb: v from row jb's own table (row jb-1 may be a pole)
    if (q.att) theta_face<T, N, true>(q, f4, R4, wdn, fl[2].vdn, Fdn);
    else theta_face<T, N, false>(q, f4, R4, wdn, fl[2].vdn, Fdn);
  }
  for (int j = jb; j < je; ++j) {
    load_row(4, j + 2);
    const int64_t ro = (int64_t)j * pitch;
    T e[N + 4];
    row_ext<T, N, 2>(fin + ro, kc, np, lane, R[2], e);
    if (act) {
      T o[N];
      if (s.c == T(0)) {
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] = s.b * R[2][i];
      } else {
        const RowGeo<T> g = geo[d.geo + j];
        const RowFlow<T> f4[4] = {fl[1], fl[2], fl[3], fl[4]};
        T R4[4][N];
#pragma unroll
        for (int m = 0; m < 4; ++m)
#pragma unroll
          for (int i = 0; i < N; ++i) R4[m][i] = R[m + 1][i];
        const bool wup = weno && (j >= 2) && (j <= nt - 4);
        T F[N + 1], Fup[N];
        if (q.att) {
          phi_faces<T, N, true>(q, fl[2].vp, e, F);
          theta_face<T, N, true>(q, f4, R4, wup, fl[2].vup, Fup);
        } else {
          phi_faces<T, N, false>(q, fl[2].vp, e, F);
          theta_face<T, N, false>(q, f4, R4, wup, fl[2].vup, Fup);
        }
#pragma unroll
        for (int i = 0; i < N; ++i) {
          const T div = (g.sup * Fup[i] - g.sdn * Fdn[i]) * g.inv_sdth + (F[i + 1] - F[i]) * g.inv_sdph;
          o[i] = s.b * R[2][i] - cdt * div;
          Fdn[i] = Fup[i];
        }
      }
      if (fn != nullptr && s.a != T(0)) {
        T f0[N];
        Vec<T>::ld(fn + ro + kc, f0);
#pragma unroll
        for (int i = 0; i < N; ++i) o[i] += s.a * f0[i];
      }
      Vec<T>::st(out + ro + kc, o);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      fl[m] = fl[m + 1];
#pragma unroll
      for (int i = 0; i < N; ++i) R[m][i] = R[m + 1][i];
    }
  }
}

// Error-free transformations in FP32 (Knuth's TwoSum; the FMA form of
// Dekker's TwoProduct): s + e equals a + b exactly, p + e equals a * b.
// The _rn intrinsics keep the compiler from contracting a product into
// these sums (an FMA there would break exactness).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// A compensated FP32 sum (Ogita, Rump and Oishi's Sum2): s + c tracks the
// exact sum of the added terms; the error of c is of order n^2 u^2 sum |x|
// for n terms (u = 2^-24), about 2e-13 sum |x| for a thread's 8 terms.
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float e;
    two_sum(s, x, s, e);
    c += e;
  }
  // x * (hi + lo), with hi + lo an FP64 value split into two floats
  __device__ __forceinline__ void add_product(float x, float hi, float lo) {
    const float p = __fmul_rn(x, hi);
    const float ep = fmaf(x, hi, -p);  // x * hi - p, exactly
    float e;
    two_sum(s, p, s, e);
    c += e + fmaf(x, lo, ep);
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// ---------------------------------------------------------------------------
// Fused RKL2 (temporal blocking): fused::K stages per launch, FP32.
//
// Rows 1 .. nt-2 are advanced in (band, strip) work items.  One warp owns a
// strip of 128 longitudes (a float4 per lane) and marches down a band of
// rows; for every RKL2 level (the two inputs delta_{j-2}, delta_{j-1} and
// the K levels it computes) the lane keeps its last two rows in registers;
// at each row step it takes one new row of the inputs and computes level m
// at the row m above, so level K leaves the pipeline K rows behind the
// loads.  The HL lanes at each edge (4 HL >= K columns) are the phi halo and
// the K rows above and below the band the theta halo: their values go stale
// from the edge inward, one point per level, and are never stored.  No block
// barrier after the start.
//
// Poles (App. A): a pole is one cell whose update needs the FP64 ring sum
// of the level below it over all longitudes, which no warp holds.  The
// operator is the same on every longitude, so the ring sums S_l[i] (row i
// counted from the pole) obey their own 1-D recurrence over the rows (the
// phi terms cancel in the sum): the K pole values of a pass follow exactly
// from the ring sums of the pass's inputs on the K rows next to each pole.
// A warp whose rows reach a pole evaluates that recurrence in FP64 first
// (pole_values), then takes the pole value at every level on the pole row
// instead of computing it, and writes the pole row of the outputs for its
// columns.  The ring sums come from per-strip partials: each warp that
// writes one of the K rows next to a pole adds up its columns of both
// outputs (compensated FP32, then FP64) for the next launch; before the
// first launch of a step ring_sums_kernel forms them for stage 1's output
// and for G.
// HBM traffic per launch: read delta_{j-2}, delta_{j-1}, G, write two
// increments: 20 B per cell per K stages instead of 16 B per stage.
// ---------------------------------------------------------------------------
namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// Asynchronous global -> shared copies (per lane, its own slots): 16 bytes
// when the four columns are contiguous and aligned, else four 4-byte copies.
__device__ __forceinline__ void async_cols(float4* dst, const float* row, int c0, int np, bool vec) {
  const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  if (vec) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(row + c0) : "memory");
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int c = c0 + e;
      c = c >= np ? c - np : c;
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa + 4 * e), "l"(row + c) : "memory");
    }
  }
}
// The 16-byte copy of async_cols issued only when `on` (a predicate, no branch).
__device__ __forceinline__ void async_vec_if(float4* dst, const float* src, bool on) {
  const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(sa),
      "l"(src), "r"((int)on)
      : "memory");
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One level update of a lane's 4 points; l/r neighbours across lanes.
// The 5-point operator and the increment-form RKL2 combination are folded
// into per-(row, level) coefficients
//   o = a0 c + a1 up + a2 dn + a3 (l + r) + nu d2 + gsum G,
//   a1..a3 = mu~ nu dt (cN, cS, cE),  a0 = mu + mu~ nu dt cC,
//   cC = -(cN + cS + 2 cE)
// (the same stage as rkl2_stage_kernel, other rounding and summation order), evaluated on (x, y) and
// (z, w) pairs with the packed f32x2 FMA: the same IEEE operations per
// element as the scalar forms (point_update below).  A row's coefficients
// for all K levels are formed once per row by the warp, one per lane, and
// read back as pairs ka = (a1, a1, a2, a2), kb = (a3, a3, a0, a0).
struct LevelNG {  // per-level constants, each duplicated into a pair
  float2 nu, gs;
};

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

__device__ __forceinline__ float4 level_update(const LevelNG& q, float4 ka, float4 kb, float4 c, float4 up,
                                               float4 dn, float4 d2, float4 gv) {
  const float l = __shfl_up_sync(0xffffffffu, c.w, 1);
  const float r = __shfl_down_sync(0xffffffffu, c.x, 1);
  const float2 h01 = make_float2(l + c.y, c.x + c.z);
  const float2 h23 = make_float2(c.y + c.w, c.z + r);
  float2 o01 = __fmul2_rn(q.gs, lo2(gv));
  float2 o23 = __fmul2_rn(q.gs, hi2(gv));
  o01 = __ffma2_rn(q.nu, lo2(d2), o01);
  o23 = __ffma2_rn(q.nu, hi2(d2), o23);
  o01 = __ffma2_rn(lo2(kb), h01, o01);
  o23 = __ffma2_rn(lo2(kb), h23, o23);
  o01 = __ffma2_rn(lo2(ka), lo2(up), o01);
  o23 = __ffma2_rn(lo2(ka), hi2(up), o23);
  o01 = __ffma2_rn(hi2(kb), lo2(c), o01);
  o23 = __ffma2_rn(hi2(kb), hi2(c), o23);
  // dn (level m-1's row computed in this same step) enters last: one FMA
  // per level on the chain through the K levels of a row step
  o01 = __ffma2_rn(hi2(ka), lo2(dn), o01);
  o23 = __ffma2_rn(hi2(ka), hi2(dn), o23);
  return make_float4(o01.x, o01.y, o23.x, o23.y);
}

// Lane state of the interior march.  W[l][q] holds level l (0..K-1; level 0
// is the input delta_{j-1}) at the row whose index mod 3 is q: level l's
// window holds its last three rows, and its new row replaces the one three
// rows up, which no level needs any more (so the state never moves between
// registers).  Level m is computed at row t-m; it reads level m-1 at rows
// t-m-1, t-m, t-m+1 (the last computed earlier in the same step), level m-2
// at row t-m and G at row t-m.  The inputs arrive through per-warp
// shared-memory rings filled D rows ahead by cp.async (each lane copies its
// own float4, so a lane only ever reads what it copied itself); G and the
// coefficient table sit in rings of period RG whose first MG slots are
// mirrored after the ring, so the K rows a step reads (t-1 .. t-K) are at
// fixed offsets below one base slot: no per-level index arithmetic.  Every
// lane forms one of the K x 4 level coefficients of each new row (level
// lane/4, coefficient lane mod 4) from the row's geometry, prefetched from
// global memory one row ahead.
struct March {
  float4 W[fused::K][3];
  float4 a_prev;             // delta_{j-2} at row t-1
  float4 *rc, *ra, *rg;      // rings: C, A (D rows), G (GSLOTS rows); this lane's slot 0
  float4* tab;               // coefficient table: GSLOTS rows x K levels x (ka, kb)
  const float* geo;          // this lane's geometry component (cN, cS, cE or cC) of row 0
  const float* pole;         // pole values of levels 1..K: north at [0..K), south at [K..2K)
  double* part_out;          // ring-sum partials for the next launch (this realization, output buffer)
  const float *nC, *nA, *nG; // this lane's columns of the inputs at the next row to request
  float gnext;               // that component of the next row to tabulate
  float kmul, kadd;          // this lane's coefficient: kmul * geometry + kadd
  int s;                     // ring slot of the current row t (t mod RG)
  int rmax;                  // last row that exists and is loaded (min(t_end, nt-1))
  int strip, ns;             // this work item's strip, strips per ring
  LevelNG lv[fused::K];      // per-level constants (registers)
};

// Partials layout of one realization (doubles, at desc.poff): ring sums of
// the launch inputs C = delta_{j-1} and A = delta_{j-2} on rows 1..K from
// each pole, per strip, in two buffers (the launch reads one and fills the
// other for the next), then those of G.
__host__ __device__ constexpr int64_t part_io(int buf, int pole, int arr, int row, int strip, int ns) {
  return ((((int64_t)buf * 2 + pole) * 2 + arr) * fused::K + (row - 1)) * ns + strip;
}
__host__ __device__ constexpr int64_t part_g(int pole, int row, int strip, int ns) {
  return ((int64_t)8 * fused::K + (int64_t)pole * fused::K + (row - 1)) * ns + strip;
}

// Warp sum of compensated partials (s, c); every lane returns the total.
__device__ __forceinline__ double warp_csum(CSum v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, v.s, o), c2 = __shfl_xor_sync(0xffffffffu, v.c, o);
    float e;
    two_sum(v.s, s2, v.s, e);
    v.c += c2 + e;
  }
  return v.value();
}

// The pole values P_1 .. P_kk of one pole for this launch (written to
// out[0..kk)), from the ring sums of the inputs: App. A's cap update with the
// FP64 ring sum, and the ring sums S_m[i] of the rows i = 1 .. kk-m from
// the pole by the ring-summed stage (the phi neighbours cancel:
// sum_k (l + r) = 2 S).  Lane i < K carries row i+1.  Returns P_kk in FP64.
__device__ double pole_values(bool north, const RealDesc& d, const StepParam& p, const Coef<float>* coef, int j0,
                              int kk, const RowGeo<float>* geo, const ShapeConst& shc, const float* gC,
                              const float* gA, const float* gG, bool zero_m2, const double* part, int pin,
                              float* out, int lane) {
  using namespace fused;
  const int ns = n_strips(d.np), pole = north ? 0 : 1;
  const int g0 = north ? 0 : d.nt - 1, dir = north ? 1 : -1;
  // lane q < 3K: array q / K (C, A, G) on row 1 + q % K, summed over the strips in order
  double sum = 0.0;
  if (lane < 3 * K) {
    const int a = lane / K, i = 1 + lane % K;
    const double* src = part + (a < 2 ? part_io(pin, pole, a, i, 0, ns) : part_g(pole, i, 0, ns));
    if (!(a == 1 && zero_m2))
      for (int s = 0; s < ns; ++s) sum += src[s];
  }
  const int q = lane < K ? lane : K - 1;
  double s1 = __shfl_sync(0xffffffffu, sum, q);          // S_{m-1}[q+1]
  double s2 = __shfl_sync(0xffffffffu, sum, K + q);      // S_{m-2}[q+1]
  const double sg = __shfl_sync(0xffffffffu, sum, 2 * K + q);
  const RowGeo<float> g = geo[d.geo + g0 + dir * (q + 1)];
  const double cp = north ? g.cN : g.cS;   // the neighbour towards the pole
  const double ca = north ? g.cS : g.cN;   // the neighbour away from it
  const double cc = double(g.cC) + 2.0 * double(g.cE);
  const double npd = d.np;
  const float nudt = float(p.nudt);
  const double lp_fac = shc.pole_diff * p.cap_nu;
  const double gp = double(gG[(int64_t)g0 * d.pitch]);
  double pm1 = double(gC[(int64_t)g0 * d.pitch]);
  double pm2 = zero_m2 ? 0.0 : double(gA[(int64_t)g0 * d.pitch]);
  double last = 0.0;
  for (int m = 1; m <= kk; ++m) {
    const Coef<float> cf = coef[p.coef + j0 + m - 1];
    const double ring = __shfl_sync(0xffffffffu, s1, 0);  // S_{m-1}[1]
    last = double(cf.mu) * pm1 + double(cf.nu) * pm2 +
           double(cf.mut) * double(nudt) * (lp_fac * (ring - npd * pm1)) + double(cf.gsum) * gp;
    const float pv = float(last);
    double up = __shfl_up_sync(0xffffffffu, s1, 1);
    const double dn = __shfl_down_sync(0xffffffffu, s1, 1);
    if (lane == 0) up = npd * pm1;
    const double md = double(cf.mut) * double(nudt);
    const double sn = double(cf.mu) * s1 + double(cf.nu) * s2 + md * (cp * up + ca * dn + cc * s1) +
                      double(cf.gsum) * sg;
    s2 = s1;
    s1 = sn;
    pm2 = pm1;
    pm1 = double(pv);
    if (lane == 0) out[m - 1] = pv;
  }
  return last;
}

// Issue the asynchronous copies of row r's inputs into the rings (one commit
// group; empty past the last loaded row, which keeps the group count
// uniform) and advance the row pointers.  xs = r mod RG, the row's G slot
// (mirrored below MG).  VEC: one predicated 16-byte copy per array.
template <bool VEC>
__device__ __forceinline__ void march_issue(March& S, int r, int xs, int pitch, int np, int col, bool zero_m2) {
  using namespace fused;
  const int sl = (r & (D - 1)) * LANES;
  const bool on = r <= S.rmax;
  if (VEC) {
    async_vec_if(S.rc + sl, S.nC, on);
    async_vec_if(S.ra + sl, S.nA, on && !zero_m2);
    async_vec_if(S.rg + xs * LANES, S.nG, on);
    async_vec_if(S.rg + (xs + RG) * LANES, S.nG, on && xs < MG);
  } else if (on) {
    async_cols(S.rc + sl, S.nC - col, col, np, false);
    if (!zero_m2) async_cols(S.ra + sl, S.nA - col, col, np, false);
    async_cols(S.rg + xs * LANES, S.nG - col, col, np, false);
    if (xs < MG) async_cols(S.rg + (xs + RG) * LANES, S.nG - col, col, np, false);
  }
  async_commit();
  S.nC += pitch;
  S.nA += pitch;
  S.nG += pitch;
}

// One row step t (phase P = t mod 3).  FULL: all K levels run (kk == K).
// EDGE: a step near a pole: level m takes the pole value where it sits on
// a pole row (t - m == 0 or nt - 1), and an output row among the K next to
// a pole adds its strip's ring-sum partials for the next launch.  Rows above
// the first loaded one (t - m < tmin during the first K steps of a band
// away from the poles) and rows past the south pole are computed from stale
// ring slots and zero windows; they only feed levels at rows that never
// reach an output.
template <int P, bool FULL, bool VEC, bool EDGE>
__device__ __forceinline__ void march_row(March& S, int t, int kk, int nt, int pitch, int np, int col,
                                          bool zero_m2, int J0, bool fin, float* oA, float* oC, float* Bs,
                                          bool lane_out, int n_out, bool& bad, int lane) {
  using namespace fused;
  // request row t+D-1 (into the C/A slots of row t-1, already consumed),
  // then wait until row t has landed: D groups are in flight at most
  {
    int xs = S.s + (D - 1);
    xs = xs >= RG ? xs - RG : xs;
    march_issue<VEC>(S, t + D - 1, xs, pitch, np, col, zero_m2);
  }
  async_wait<D - 1>();
  const int cs = (t & (D - 1)) * LANES;
  S.W[0][P] = S.rc[cs];
  const float4 a_t = zero_m2 ? make_float4(0.f, 0.f, 0.f, 0.f) : S.ra[cs];
  const int P0 = S.s >= K ? S.s : S.s + RG;     // row t-m of G and the table: slot P0 - m
  const float4* gb = S.rg + P0 * LANES;
  const float4* kb = S.tab + P0 * (2 * K);
  float4 top = make_float4(0.f, 0.f, 0.f, 0.f);  // level K at row t-K
#pragma unroll
  for (int m = 1; m <= K; ++m) {
    if (FULL || m <= kk) {
      const int sc = ((P - m) % 3 + 3) % 3;      // slot of row t-m
      const int su = ((P - m - 1) % 3 + 3) % 3;  // row t-m-1
      const int sd = ((P - m + 1) % 3 + 3) % 3;  // row t-m+1 (level m-1's newest)
      const float4 d2 = m == 1 ? S.a_prev : S.W[m - 2][sc];
      const float4 gv = gb[-m * LANES];
      const float4* kr = kb - m * (2 * K) + 2 * (m - 1);
      float4 o = level_update(S.lv[m - 1], kr[0], kr[1], S.W[m - 1][sc], S.W[m - 1][su], S.W[m - 1][sd], d2, gv);
      if (EDGE) {
        if (t - m == 0) {
          const float v = S.pole[m - 1];
          o = make_float4(v, v, v, v);
        } else if (t - m == nt - 1) {
          const float v = S.pole[K + m - 1];
          o = make_float4(v, v, v, v);
        }
      }
      if (m < K) S.W[m][sc] = o;
      else top = o;
    }
  }
  S.a_prev = a_t;
  // leave the pipeline: level kk (and kk-1) at row t - kk (always < J1)
  const int orow = t - (FULL ? K : kk);
  // slots are compile-time (unrolled m, template P) so the state stays in registers
  float4 lk = top, lk1 = S.W[K - 1][((P - K) % 3 + 3) % 3];
  if (!FULL) {
#pragma unroll
    for (int m = 1; m < K; ++m)
      if (m == kk) {
        lk = S.W[m][((P - m) % 3 + 3) % 3];
        lk1 = S.W[m - 1][((P - m) % 3 + 3) % 3];
      }
  }
  if (orow >= J0 && lane_out) {
    const int64_t go = (int64_t)orow * pitch + col;
    if (fin) {
      if (n_out == 4 && VEC) {
        float4 b = ld4(Bs + go);
        b.x += lk.x; b.y += lk.y; b.z += lk.z; b.w += lk.w;
        bad |= !isfinite(b.x) || !isfinite(b.y) || !isfinite(b.z) || !isfinite(b.w);
        st4(Bs + go, b);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (e < n_out) {
            int c = col + e;
            c = c >= np ? c - np : c;
            const float x = Bs[(int64_t)orow * pitch + c] + (e == 0 ? lk.x : e == 1 ? lk.y : e == 2 ? lk.z : lk.w);
            bad |= !isfinite(x);
            Bs[(int64_t)orow * pitch + c] = x;
          }
        }
      }
    } else if (n_out == 4 && VEC) {
      st4(oC + go, lk);
      st4(oA + go, lk1);
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        if (e < n_out) {
          int c = col + e;
          c = c >= np ? c - np : c;
          oC[(int64_t)orow * pitch + c] = e == 0 ? lk.x : e == 1 ? lk.y : e == 2 ? lk.z : lk.w;
          oA[(int64_t)orow * pitch + c] = e == 0 ? lk1.x : e == 1 ? lk1.y : e == 2 ? lk1.z : lk1.w;
        }
      }
    }
  }
  // ring-sum partials of the rows next to a pole (uniform over the warp)
  if (EDGE && !fin && orow >= J0 && (orow <= K || orow >= nt - 1 - K)) {
    CSum sc, sa;
    const float vc[4] = {lk.x, lk.y, lk.z, lk.w}, va[4] = {lk1.x, lk1.y, lk1.z, lk1.w};
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (e < n_out) {
        sc.add(vc[e]);
        sa.add(va[e]);
      }
    const double tc = warp_csum(sc), ta = warp_csum(sa);
    if (lane == 0) {
      const int pole = orow <= K ? 0 : 1, row = orow <= K ? orow : nt - 1 - orow;
      S.part_out[part_io(0, pole, 0, row, S.strip, S.ns)] = tc;
      S.part_out[part_io(0, pole, 1, row, S.strip, S.ns)] = ta;
    }
  }
  // row t's coefficients (first read at step t+1) into slot t mod RG (and its mirror)
  {
    const float v = fmaf(S.kmul, S.gnext, S.kadd);
    float2* tb = reinterpret_cast<float2*>(S.tab) + lane;
    if (4 * K == LANES || lane < 4 * K) {
      tb[S.s * (4 * K)] = make_float2(v, v);
      // the mirror copy, or a spare slot after the ring (no branch)
      tb[(S.s < MG ? S.s + RG : GSLOTS) * (4 * K)] = make_float2(v, v);
    }
    S.gnext = S.geo[(int64_t)min(t + 1, nt - 1) * (sizeof(RowGeo<float>) / sizeof(float))];
  }
  S.s = S.s + 1 == RG ? 0 : S.s + 1;
  __syncwarp();
}

// Row steps t0 .. t1-1, unrolled by 3 so that the window phase t mod 3 is a
// template argument.
template <bool FULL, bool VEC, bool EDGE>
__device__ __forceinline__ void march_run(March& S, int t0, int t1, int kk, int nt, int pitch, int np, int col,
                                          bool zero_m2, int J0, bool fin, float* oA, float* oC, float* Bs,
                                          bool lane_out, int n_out, bool& bad, int lane) {
#define SFT_MARCH(PH, TT)                                                                                    \
  march_row<PH, FULL, VEC, EDGE>(S, TT, kk, nt, pitch, np, col, zero_m2, J0, fin, oA, oC, Bs, lane_out, n_out, \
                                 bad, lane)
  int t = t0;
  const int ph = t % 3;
  if (t < t1 && ph == 1) {
    SFT_MARCH(1, t);
    ++t;
  }
  if (t < t1 && ph != 0) {
    SFT_MARCH(2, t);
    ++t;
  }
  for (; t + 2 < t1; t += 3) {
    SFT_MARCH(0, t);
    SFT_MARCH(1, t + 1);
    SFT_MARCH(2, t + 2);
  }
  if (t < t1) {
    SFT_MARCH(0, t);
    ++t;
  }
  if (t < t1) SFT_MARCH(1, t);
#undef SFT_MARCH
}

// The row loop of one work item: rows tmin..t_end.  The steps near a pole
// (where a level can sit on the pole row, or an output row is one of the K
// next to a pole) run the EDGE instance: the first kk + K + 1 steps of the
// band starting at the north pole, the steps from nt-1-K+kk of a band
// reaching the south pole.
template <bool FULL, bool VEC>
__device__ __forceinline__ void march_band(March& S, int tmin, int t_end, int kk, int nt, int pitch, int np,
                                           int col, bool zero_m2, int J0, bool fin, float* oA, float* oC,
                                           float* Bs, bool lane_out, int n_out, bool& bad, int lane) {
  using namespace fused;
  S.s = tmin % RG;
  for (int i = 0; i < D - 1; ++i) {  // D-1 rows of lookahead before the first step
    int xs = S.s + i;
    xs = xs >= RG ? xs - RG : xs;
    march_issue<VEC>(S, tmin + i, xs, pitch, np, col, zero_m2);
  }
  S.gnext = S.geo[(int64_t)tmin * (sizeof(RowGeo<float>) / sizeof(float))];
  const int n_end = tmin == 0 ? min(kk + K + 1, t_end + 1) : tmin;
  const int s_beg = t_end >= nt - 1 - K + kk ? max(n_end, nt - 1 - K + kk) : t_end + 1;
#define SFT_RUN(E, A, B_)                                                                                  \
  march_run<FULL, VEC, E>(S, A, B_, kk, nt, pitch, np, col, zero_m2, J0, fin, oA, oC, Bs, lane_out, n_out, bad, \
                          lane)
  SFT_RUN(true, tmin, n_end);
  SFT_RUN(false, n_end, s_beg);
  SFT_RUN(true, s_beg, t_end + 1);
#undef SFT_RUN
}

}  // namespace

__global__ void __launch_bounds__(fused::THREADS, fused::MIN_BLOCKS)
rkl2_fused_kernel(const Tile* __restrict__ tiles, const RealDesc* __restrict__ rd,
                  const StepParam* __restrict__ sp, const RowGeo<float>* __restrict__ geo,
                  const ShapeConst* __restrict__ shc, const Coef<float>* __restrict__ coef,
                  float* __restrict__ B, const float* __restrict__ G, const float* __restrict__ Dm2,
                  const float* __restrict__ Dm1, float* __restrict__ Om2, float* __restrict__ Om1,
                  double* __restrict__ part, int pin, int j0, int* __restrict__ status) {
  using namespace fused;
  __shared__ Coef<float> s_cf[K];
  const Tile tl = tiles[blockIdx.x];
  const RealDesc d = rd[tl.r];
  const StepParam p = sp[tl.r];
  if (j0 > p.s) return;  // uniform over the block
  const int kk = min(K, p.s - j0 + 1);  // levels of this realization in this launch
  if (threadIdx.x < K) s_cf[threadIdx.x] = coef[p.coef + j0 + min((int)threadIdx.x, kk - 1)];
  __syncthreads();
  const bool fin = j0 + kk - 1 == p.s;  // the launch ends the realization's super-step
  const float nudt = float(p.nudt);
  const int pitch = d.pitch, np = d.np, nt = d.nt;
  const float* gG = G + d.woff;
  const float* gA = Dm2 + d.woff;  // delta_{j0-2}
  const float* gC = Dm1 + d.woff;  // delta_{j0-1}
  float* oA = Om2 + d.woff;
  float* oC = Om1 + d.woff;
  float* Bs = B + d.off;
  const bool zero_m2 = j0 == 2;  // delta_0 = 0

  // warp w of the block marches work item (tl.j0 + w) = (band, strip)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ns = n_strips(np);
  const int band = d.band;
  const int item = tl.j0 + warp;
  if (item >= n_bands(nt, band) * ns) return;  // whole warp
  const int strip = item % ns;
  const int J0 = 1 + (item / ns) * band;
  const int J1 = min(J0 + band, nt - 1);
  int col = (strip * STRIP - 4 * HL + 4 * lane) % np;  // first of the lane's 4 columns, periodic
  col = col < 0 ? col + np : col;
  const bool vec = (np & 3) == 0;
  // output: lanes HL..31-HL, columns strip*STRIP .. +STRIP-1 that are < np
  const int first_out = strip * STRIP + 4 * (lane - HL);
  const bool lane_out = lane >= HL && lane < LANES - HL && first_out < np;
  const int n_out = lane_out ? min(4, np - first_out) : 0;
  extern __shared__ __align__(16) float4 rings[];
  const int tmin = max(J0 - K, 0);  // first row loaded
  const int t_end = J1 - 1 + kk;    // last row step (rows past nt-1 are not loaded)
#ifdef SFT_DEBUG
  // every row the band loads or writes lies in [tmin, nt-1]; a band or a
  // column outside the realization skips the work item (whole warp: the
  // march shuffles across lanes) after its check is recorded
  const bool dbg_bad = dbg_check(DBG_FUSED_FIRST, tmin, 0, nt - 1) != tmin ||
                       dbg_check(DBG_FUSED_LAST, J1, J0, nt - 1) != J1 ||
                       dbg_check(DBG_FUSED_COL, col, 0, vec ? np - 4 : np - 1) != col;
  if (__any_sync(0xffffffffu, dbg_bad)) return;
#endif
  March S;
  S.rc = rings + warp * RING_F4 + lane;
  S.ra = S.rc + D * LANES;
  S.rg = S.ra + D * LANES;
  S.tab = rings + WARPS * RING_F4 + warp * TAB_F4;
  float* spole = reinterpret_cast<float*>(rings + WARPS * (RING_F4 + TAB_F4)) + warp * 2 * K;
  S.pole = spole;
  S.geo = reinterpret_cast<const float*>(geo + d.geo) + (lane & 3);
  S.rmax = min(t_end, nt - 1);
  S.strip = strip;
  S.ns = ns;
  S.part_out = part + d.poff + part_io(1 - pin, 0, 0, 1, 0, ns);
  // pole values of this launch for the poles the band's rows reach (a level
  // on the pole row) or whose pole row the band owns (the first band the
  // north pole, the last band the south pole): the owner writes the pole
  // row of the outputs for this strip's columns
  for (int pole = 0; pole < 2; ++pole) {
    const bool north = pole == 0;
    const bool own = north ? J0 == 1 : J1 == nt - 1;
    if (!own && (north ? tmin != 0 : t_end < nt)) continue;
    const double last = pole_values(north, d, p, coef, j0, kk, geo, shc[d.shape], gC, gA, gG, zero_m2,
                                    part + d.poff, pin, spole + pole * K, lane);
    __syncwarp();
    if (!own) continue;
    const float pk = spole[pole * K + kk - 1];
    const float pk1 = kk >= 2 ? spole[pole * K + kk - 2] : gC[(int64_t)(north ? 0 : nt - 1) * pitch];
    const int64_t ro = (int64_t)(north ? 0 : nt - 1) * pitch;
    for (int e = 0; e < n_out; ++e) {
      const int c = first_out + e;
      if (fin) {
        const float v = float(double(Bs[ro + c]) + last);
        if (!isfinite(v)) atomicOr(status, 1);
        Bs[ro + c] = v;
      } else {
        oC[ro + c] = pk;
        oA[ro + c] = pk1;
      }
    }
  }
  {
    // lane = 4 (level - 1) + coefficient: a1 = md cN, a2 = md cS, a3 = md cE, a0 = mu + md cC
    const Coef<float> c = s_cf[min(lane >> 2, K - 1)];
    S.kmul = c.mut * nudt;
    S.kadd = (lane & 3) == 3 ? c.mu : 0.f;
  }
#pragma unroll
  for (int m = 0; m < K; ++m) {
    const Coef<float> c = s_cf[m];
    S.lv[m] = LevelNG{make_float2(c.nu, c.nu), make_float2(c.gsum, c.gsum)};
  }
#pragma unroll
  for (int l = 0; l < K; ++l)
#pragma unroll
    for (int q = 0; q < 3; ++q) S.W[l][q] = make_float4(0.f, 0.f, 0.f, 0.f);
  S.a_prev = make_float4(0.f, 0.f, 0.f, 0.f);
  S.nC = gC + (int64_t)tmin * pitch + col;
  S.nA = gA + (int64_t)tmin * pitch + col;
  S.nG = gG + (int64_t)tmin * pitch + col;
  bool bad = false;
  // (kk == K, np % 4 == 0) is the hot instance; the others serve the last
  // launch of a realization and grids whose rows are not float4-aligned
#define SFT_BAND(F, V)                                                                                          \
  march_band<F, V>(S, tmin, t_end, kk, nt, pitch, np, col, zero_m2, J0, fin, oA, oC, Bs, lane_out, n_out, bad, \
                   lane)
  if (vec) {
    if (kk == K) SFT_BAND(true, true);
    else SFT_BAND(false, true);
  } else {
    if (kk == K) SFT_BAND(true, false);
    else SFT_BAND(false, false);
  }
#undef SFT_BAND
  async_wait<0>();  // no copy outlives the block
  if (bad) atomicOr(status, 1);
}

// Ring-sum partials of the rows 1..K from each pole for the first fused
// launch of a step: of stage 1's output delta_1 (input C of that launch,
// buffer 0) and of G (all launches of the step).  One block per (pole
// tile, row): tiles hold a north (kind 1) and a south (kind 2) tile per
// realization; warp w forms strips w, w+4, ... over the same columns as the
// interior's work items.
__global__ void __launch_bounds__(fused::THREADS)
ring_sums_kernel(const Tile* __restrict__ tiles, const RealDesc* __restrict__ rd, const float* __restrict__ D1,
                 const float* __restrict__ G, double* __restrict__ part) {
  using namespace fused;
  const Tile tl = tiles[blockIdx.x / K];
  const int pole = (tl.kind & 3) == 1 ? 0 : 1, row = 1 + blockIdx.x % K;
  const RealDesc d = rd[tl.r];
  const int ns = n_strips(d.np);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ro = d.woff + (int64_t)(pole == 0 ? row : d.nt - 1 - row) * d.pitch;
  for (int s = warp; s < ns; s += WARPS) {
    CSum sc, sg;
    if (lane < LANES - 2 * HL) {
      const int c0 = s * STRIP + 4 * lane;
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (c0 + e < d.np) {
          sc.add(D1[ro + c0 + e]);
          sg.add(G[ro + c0 + e]);
        }
    }
    const double tc = warp_csum(sc), tg = warp_csum(sg);
    if (lane == 0) {
      part[d.poff + part_io(0, pole, 0, row, s, ns)] = tc;
      part[d.poff + part_g(pole, row, s, ns)] = tg;
    }
  }
}

cudaError_t prepare_rkl2_fused() {
  return cudaFuncSetAttribute(rkl2_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)fused::kSmemBytes);
}

cudaError_t launch_ring_sums(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                             const float* D1, const float* G, double* part) {
  if (n_tiles <= 0) return cudaSuccess;
  ring_sums_kernel<<<n_tiles * fused::K, fused::THREADS, 0, st>>>(tiles, rd, D1, G, part);
  return cudaGetLastError();
}

cudaError_t launch_rkl2_fused(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                              const StepParam* sp, const RowGeo<float>* geo, const ShapeConst* shc,
                              const Coef<float>* coef, float* B, const float* G, const float* Dm2,
                              const float* Dm1, float* Om2, float* Om1, double* part, int pin, int j0,
                              int* status) {
  if (n_tiles <= 0) return cudaSuccess;
  rkl2_fused_kernel<<<n_tiles, fused::THREADS, fused::kSmemBytes, st>>>(tiles, rd, sp, geo, shc, coef, B, G, Dm2,
                                                                         Dm1, Om2, Om1, part, pin, j0, status);
  return cudaGetLastError();
}

template <typename T>
__global__ void fix_poles_kernel(const RealDesc* __restrict__ rd, T* __restrict__ state, int only_r) {
  const int r = only_r >= 0 ? only_r : blockIdx.x >> 1;
  const RealDesc d = rd[r];
  const int jp = (blockIdx.x & 1) ? d.nt - 1 : 0;
  T* row = state + d.off + (int64_t)jp * d.pitch;
  const T v = row[0];
  __syncthreads();
  for (int k = threadIdx.x + 1; k < d.np; k += blockDim.x) row[k] = v;
}

// ---------------------------------------------------------------------------
// Reductions (FP64 accumulation)
// ---------------------------------------------------------------------------
namespace {

template <typename T>
__device__ __forceinline__ T ldT(const void* p, int64_t i) {
  return static_cast<const T*>(p)[i];
}

// Eq. (data_assim_f): F = mu^alpha_mu if mu > mu_lim and |lat| < lat_lim.
template <typename T>
__device__ __forceinline__ T assim_weight(T mu, double lat, const double* w) {
  if (!(double(mu) > w[1]) || !(fabs(lat) < w[2])) return T(0);
  return pow(mu, T(w[0]));
}

__device__ double block_min(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  double t = sm[0];
  for (int i = 1; i < (int)(blockDim.x >> 5); ++i) t = fmin(t, sm[i]);
  return t;
}

}  // namespace

template <typename T>
__global__ void __launch_bounds__(kThreads)
reduce_kernel(int mode, const RedTile* __restrict__ tiles, const RealDesc* __restrict__ rd,
              const RowGeoD* __restrict__ geod, const double* __restrict__ cosp,
              const double* __restrict__ sinp, const float4* __restrict__ csf, const T* __restrict__ state,
              double lat_cut, AssimArgs aa, double* __restrict__ partials) {
  __shared__ double sm[kThreads / 32];
  const RedTile tl = tiles[blockIdx.x];
  const RealDesc d = rd[tl.r];
  const T* b = state + d.off;
  int j0 = tl.j0, j1 = tl.j1;
  SFT_DCHECK(DBG_RED_ROWS, j0, 0, d.nt);
  SFT_DCHECK(DBG_RED_ROWS, j1, j0, d.nt);
  double acc[11];
#pragma unroll
  for (int f = 0; f < 11; ++f) acc[f] = 0.0;
  double mn = INFINITY, mx = -INFINITY, amn = INFINITY;
  const double* w = aa.wpar ? aa.wpar + 4 * tl.r : nullptr;
  const int64_t obase = aa.obs_off ? aa.obs_off[tl.r] : 0;
  T tmn = T(INFINITY), tmx = T(-INFINITY), tamn = T(INFINITY);
  for (int j = j0; j < j1; ++j) {
    const RowGeoD gd = geod[d.geo + j];
    const bool pole = (j == 0) || (j == d.nt - 1);
    const T* row = b + (int64_t)j * d.pitch;
    if (mode == RED_DIAG) {
      // Row constants (area, cos, sin, latitude) multiply this thread's row
      // sums once: per cell only sum x, sum max(x, 0), sum x cos(phi) and
      // sum x sin(phi) run in FP64 (min / max are exact in T).
      double rs = 0.0, rp = 0.0, rc = 0.0, rn = 0.0;
      if constexpr (sizeof(T) == 4) {
        // FP32 state: the thread's row sums as compensated FP32 sums (GB300's
        // FP64 pipe is narrow), cos / sin phi as hi + lo float pairs; FP64
        // from the row sums on
        CSum ss, sp, sc, sn;
        for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
          const float bv = float(row[k]);
          if (!isfinite(bv)) {
            acc[10] += 1.0;
            continue;
          }
          const float4 cs = csf[d.col + k];  // (cos hi, cos lo, sin hi, sin lo)
          ss.add(bv);
          sp.add(bv > 0.f ? bv : 0.f);
          sc.add_product(bv, cs.x, cs.y);
          sn.add_product(bv, cs.z, cs.w);
          tmn = bv < tmn ? bv : tmn;
          tmx = bv > tmx ? bv : tmx;
          const float ab = bv < 0.f ? -bv : bv;
          tamn = ab < tamn ? ab : tamn;
        }
        rs = ss.value();
        rp = sp.value();
        rc = sc.value();
        rn = sn.value();
      } else {
        for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
          const T bv = row[k];
          if (!isfinite(bv)) {
            acc[10] += 1.0;
            continue;
          }
          const double x = double(bv);
          rs += x;
          rp += bv > T(0) ? x : 0.0;
          rc = fma(x, cosp[d.col + k], rc);
          rn = fma(x, sinp[d.col + k], rn);
          tmn = bv < tmn ? bv : tmn;
          tmx = bv > tmx ? bv : tmx;
          const T ab = bv < T(0) ? -bv : bv;
          tamn = ab < tamn ? ab : tamn;
        }
      }
      acc[0] += gd.area * rs;
      acc[1] += gd.area * rp;
      acc[2] += gd.area * (rs - rp);
      if (gd.lat >= lat_cut - 1e-12) {
        acc[3] += gd.area * rs;
        if (threadIdx.x == 0) acc[5] += gd.area * d.np;
      }
      if (gd.lat <= -lat_cut + 1e-12) {
        acc[4] += gd.area * rs;
        if (threadIdx.x == 0) acc[6] += gd.area * d.np;
      }
      acc[7] += gd.area * gd.cos_t * rs;
      acc[8] += gd.area * gd.sin_t * rc;
      acc[9] += gd.area * gd.sin_t * rn;
      continue;
    }
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
      const T bv = row[k];
      T x;
      if (mode == RED_ASSIM) {
        const int kk = pole ? 0 : k;
        const int64_t oi = obase + (int64_t)j * d.np + kk;
        const T F = assim_weight<T>(ldT<T>(aa.mu, oi), gd.lat, w);
        x = F * (ldT<T>(aa.obs, oi) - bv);
      } else {
        x = bv;
      }
      const double ax = gd.area * double(x);
      if (x > T(0)) acc[0] += ax;
      if (x < T(0)) acc[1] += ax;
    }
  }
  mn = double(tmn);
  mx = double(tmx);
  amn = double(tamn);
  double* out = partials + (int64_t)blockIdx.x * kDiagFields;
  const int nf = mode == RED_DIAG ? 11 : 2;
  for (int f = 0; f < nf; ++f) {
    const double t = block_sum(acc[f], sm);
    if (threadIdx.x == 0) out[f] = t;
  }
  if (mode == RED_DIAG) {
    const double a = block_min(mn, sm);
    if (threadIdx.x == 0) out[11] = a;
    const double c = -block_min(-mx, sm);
    if (threadIdx.x == 0) out[12] = c;
    const double e = block_min(amn, sm);
    if (threadIdx.x == 0) out[13] = e;
  }
}

// One block per realization: fold its tiles' partials in a fixed order.
// RED_DIAG: out[r*kDiagFields + f].  RED_ASSIM / RED_BALANCE: out[r*4 + ...] =
// {phi+, phi-, factor for x > 0, factor for x <= 0} (Eq. fluxbal).
__global__ void fold_kernel(int mode, const int* __restrict__ tile_start,
                            const double* __restrict__ partials, const double* __restrict__ wpar,
                            double* __restrict__ out) {
  __shared__ double sm[kThreads / 32];
  const int r = blockIdx.x;
  const int t0 = tile_start[r], t1 = tile_start[r + 1];
  const int nf = mode == RED_DIAG ? kDiagFields : 2;
  double res[kDiagFields];
  for (int f = 0; f < nf; ++f) {
    const bool is_min = mode == RED_DIAG && (f == 11 || f == 13);
    const bool is_max = mode == RED_DIAG && f == 12;
    double v = is_min ? INFINITY : (is_max ? -INFINITY : 0.0);
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      const double x = partials[(int64_t)t * kDiagFields + f];
      v = is_min ? fmin(v, x) : (is_max ? fmax(v, x) : v + x);
    }
    if (is_min) res[f] = block_min(v, sm);
    else if (is_max) res[f] = -block_min(-v, sm);
    else res[f] = block_sum(v, sm);
  }
  if (threadIdx.x != 0) return;
  if (mode == RED_DIAG) {
    for (int f = 0; f < kDiagFields; ++f) out[(int64_t)r * kDiagFields + f] = res[f];
    return;
  }
  const double pp = res[0], pm = res[1];
  double fp = 1.0, fm = 1.0;
  const bool balance = mode == RED_BALANCE || (wpar && wpar[4 * r + 3] != 0.0);
  if (balance && pp != 0.0 && pm != 0.0) {
    const double ratio = fabs(pp / pm);
    fp = 1.0 / sqrt(ratio);
    fm = sqrt(ratio);
  }
  out[4 * r + 0] = pp;
  out[4 * r + 1] = pm;
  out[4 * r + 2] = fp;
  out[4 * r + 3] = fm;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
apply_kernel(int mode, const RedTile* __restrict__ tiles, const RealDesc* __restrict__ rd,
             const RowGeoD* __restrict__ geod, T* __restrict__ state, AssimArgs aa,
             const double* __restrict__ fac) {
  const RedTile tl = tiles[blockIdx.x];
  const RealDesc d = rd[tl.r];
  T* b = state + d.off;
  const T fp = T(fac[4 * tl.r + 2]), fm = T(fac[4 * tl.r + 3]);
  const double* w = aa.wpar ? aa.wpar + 4 * tl.r : nullptr;
  const int64_t obase = aa.obs_off ? aa.obs_off[tl.r] : 0;
  for (int j = tl.j0; j < tl.j1; ++j) {
    const double lat = geod[d.geo + j].lat;
    const bool pole = (j == 0) || (j == d.nt - 1);
    T* row = b + (int64_t)j * d.pitch;
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
      const T bv = row[k];
      if (mode == RED_ASSIM) {
        const int kk = pole ? 0 : k;
        const int64_t oi = obase + (int64_t)j * d.np + kk;
        const T F = assim_weight<T>(ldT<T>(aa.mu, oi), lat, w);
        const T x = F * (ldT<T>(aa.obs, oi) - bv);
        row[k] = bv + (x > T(0) ? x * fp : x * fm);
      } else {
        row[k] = bv > T(0) ? bv * fp : bv * fm;
      }
    }
  }
}


// ---------------------------------------------------------------------------
// Random flux emergence (Sec. 2.4).  Map m's normal draw of cell c is
// counter-based (no stored maps): the SplitMix64 output function (Steele, Lea
// & Flood 2014) of the states seed + (2n+1) gamma and seed + (2n+2) gamma,
// n = m N_cells + c, as two uniforms, and Box-Muller.  FP64 grids draw in
// FP64 (53-bit uniforms), FP32 grids in FP32 (24-bit uniforms).  Cell ids:
// north cap 0, interior 1 + (j-1) np + k, south cap N_cells - 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix_output(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T> __device__ __forceinline__ T rfe_normal(uint64_t seed, uint64_t n);
template <> __device__ __forceinline__ double rfe_normal<double>(uint64_t seed, uint64_t n) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t z1 = splitmix_output(seed + (2 * n + 1) * g), z2 = splitmix_output(seed + (2 * n + 2) * g);
  const double u1 = ((double)(z1 >> 11) + 0.5) * 0x1p-53, u2 = ((double)(z2 >> 11) + 0.5) * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}
template <> __device__ __forceinline__ float rfe_normal<float>(uint64_t seed, uint64_t n) {
  const uint64_t g = 0x9E3779B97F4A7C15ull;
  const uint64_t z1 = splitmix_output(seed + (2 * n + 1) * g), z2 = splitmix_output(seed + (2 * n + 2) * g);
  const float u1 = ((float)(z1 >> 40) + 0.5f) * 0x1p-24f, u2 = ((float)(z2 >> 40) + 0.5f) * 0x1p-24f;
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// FP64 positive / negative fluxes of the (unbalanced) maps m0..m0+3 of a
// realization whose window is new this step: partials[tile][2m], [2m+1]
// (Eq. fluxbal needs them per map; the factors are kept while the window is).
template <typename T>
__global__ void __launch_bounds__(kThreads)
rfe_sums_kernel(const RedTile* __restrict__ tiles, const RealDesc* __restrict__ rd,
                const RowGeoD* __restrict__ geod, const RfeStep* __restrict__ rs, double* __restrict__ partials) {
  __shared__ double sm[kThreads / 32];
  const RedTile tl = tiles[blockIdx.x];
  const RealDesc d = rd[tl.r];
  const RfeStep R = rs[tl.r];
  double acc[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) acc[f] = 0.0;
  if (R.method != 0 && R.fresh) {
    const int64_t ncell = (int64_t)(d.nt - 2) * d.np + 2;
    for (int j = tl.j0; j < tl.j1; ++j) {
      const RowGeoD gd = geod[d.geo + j];
      const bool pole = j == 0 || j == d.nt - 1;
      const double cell_area = pole ? gd.area * d.np : gd.area;  // a cap is one cell
      const double sc = R.method == 1 ? R.c / cell_area : R.c;
      for (int k = threadIdx.x; k < (pole ? 1 : d.np); k += blockDim.x) {
        const int64_t cell = pole ? (j == 0 ? 0 : ncell - 1) : 1 + (int64_t)(j - 1) * d.np + k;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const double S = sc * double(rfe_normal<T>(R.seed, (uint64_t)(R.m0 + m) * (uint64_t)ncell + cell));
          if (S > 0.0) acc[2 * m] += cell_area * S;
          else if (S < 0.0) acc[2 * m + 1] += cell_area * S;
        }
      }
    }
  }
  double* out = partials + (int64_t)blockIdx.x * kDiagFields;
#pragma unroll
  for (int f = 0; f < 8; ++f) {
    const double t = block_sum(acc[f], sm);
    if (threadIdx.x == 0) out[f] = t;
  }
}

// One block per realization: fold the tiles' partials in a fixed order and
// form Eq. (fluxbal)'s factors per map: fac[r][2m] for S > 0, [2m+1] for S <= 0.
__global__ void rfe_fold_kernel(const int* __restrict__ tile_start, const RfeStep* __restrict__ rs,
                                const double* __restrict__ partials, double* __restrict__ fac) {
  __shared__ double sm[kThreads / 32];
  const int r = blockIdx.x;
  if (rs[r].method == 0 || !rs[r].fresh) return;  // uniform over the block
  const int t0 = tile_start[r], t1 = tile_start[r + 1];
  double v[8];
  for (int f = 0; f < 8; ++f) {
    double a = 0.0;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) a += partials[(int64_t)t * kDiagFields + f];
    v[f] = block_sum(a, sm);
  }
  if (threadIdx.x != 0) return;
  for (int m = 0; m < 4; ++m) {
    const double pp = v[2 * m], pm = v[2 * m + 1];
    double fp = 1.0, fm = 1.0;
    if (pp != 0.0 && pm != 0.0) {
      const double ratio = fabs(pp / pm);
      fp = 1.0 / sqrt(ratio);
      fm = sqrt(ratio);
    }
    fac[8 * r + 2 * m] = fp;
    fac[8 * r + 2 * m + 1] = fm;
  }
}

// B += sum_m w_m S_m (balanced), phase 0 with wa, phase 1 with wb, in the
// state's precision: per map the weight times the Eq. (fluxbal) factor of
// each sign (S has the sign of its draw), per row the map scale.
template <typename T>
__global__ void __launch_bounds__(kThreads)
rfe_apply_kernel(const RedTile* __restrict__ tiles, const RealDesc* __restrict__ rd,
                 const RowGeoD* __restrict__ geod, const RfeStep* __restrict__ rs, const double* __restrict__ fac,
                 int phase, T* __restrict__ state) {
  const RedTile tl = tiles[blockIdx.x];
  const RfeStep R = rs[tl.r];
  if (R.method == 0) return;
  const RealDesc d = rd[tl.r];
  const double* w = phase == 0 ? R.wa : R.wb;
  const double* fr = fac + 8 * tl.r;
  T wp[4], wn[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    wp[m] = T(w[m] * fr[2 * m]);
    wn[m] = T(w[m] * fr[2 * m + 1]);
  }
  const int64_t ncell = (int64_t)(d.nt - 2) * d.np + 2;
  T* b = state + d.off;
  int j0 = tl.j0, j1 = tl.j1;
  SFT_DCHECK(DBG_RED_ROWS, j0, 0, d.nt);
  SFT_DCHECK(DBG_RED_ROWS, j1, j0, d.nt);
  for (int j = j0; j < j1; ++j) {
    const RowGeoD gd = geod[d.geo + j];
    const bool pole = j == 0 || j == d.nt - 1;
    const double cell_area = pole ? gd.area * d.np : gd.area;
    const T sc = T(R.method == 1 ? R.c / cell_area : R.c);
    T* row = b + (int64_t)j * d.pitch;
    for (int k = threadIdx.x; k < d.np; k += blockDim.x) {
      const int64_t cell = pole ? (j == 0 ? 0 : ncell - 1) : 1 + (int64_t)(j - 1) * d.np + k;
      T add = T(0);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (w[m] == 0.0) continue;
        const T y = rfe_normal<T>(R.seed, (uint64_t)(R.m0 + m) * (uint64_t)ncell + cell);
        add += sc * y * (y > T(0) ? wp[m] : wn[m]);
      }
      row[k] += add;
    }
  }
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_rkl2_stage(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                              const StepParam* sp, const RowGeo<T>* geo, const ShapeConst* shc,
                              const Coef<T>* coef, T* B, T* G, T* D0, T* D1, int stage,
                              int allow_final, int* status) {
  if (n_tiles <= 0) return cudaSuccess;
  rkl2_stage_kernel<T><<<n_tiles, kThreads, 0, st>>>(tiles, rd, sp, geo, shc, coef, B, G, D0, D1,
                                                     stage, allow_final, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adv_stage(int n_tiles, cudaStream_t st, const Tile* tiles, const RealDesc* rd,
                             const StepParam* sp, const RowGeo<T>* geo, const RowFlow<T>* flow,
                             const ShapeConst* shc, T* state, T* w0, T* w1, AdvStage<T> s) {
  if (n_tiles <= 0) return cudaSuccess;
  adv_stage_kernel<T><<<n_tiles, kThreads, 0, st>>>(tiles, rd, sp, geo, flow, shc, state, w0, w1, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fix_poles(int n_real, cudaStream_t st, const RealDesc* rd, T* state, int only_r) {
  const int blocks = only_r >= 0 ? 2 : 2 * n_real;
  if (blocks <= 0) return cudaSuccess;
  fix_poles_kernel<T><<<blocks, kThreads, 0, st>>>(rd, state, only_r);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce(int mode, int n_tiles, cudaStream_t st, const RedTile* tiles,
                          const RealDesc* rd, const RowGeoD* geod, const double* cosp,
                          const double* sinp, const float4* csf, const T* state, double lat_cut,
                          AssimArgs aa, double* partials) {
  if (n_tiles <= 0) return cudaSuccess;
  reduce_kernel<T><<<n_tiles, kThreads, 0, st>>>(mode, tiles, rd, geod, cosp, sinp, csf, state, lat_cut,
                                                 aa, partials);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rfe_sums(int n_tiles, cudaStream_t st, const RedTile* tiles, const RealDesc* rd,
                            const RowGeoD* geod, const RfeStep* rs, double* partials) {
  if (n_tiles <= 0) return cudaSuccess;
  rfe_sums_kernel<T><<<n_tiles, kThreads, 0, st>>>(tiles, rd, geod, rs, partials);
  return cudaGetLastError();
}

cudaError_t launch_rfe_fold(int n_real, cudaStream_t st, const int* tile_start, const RfeStep* rs,
                            const double* partials, double* fac) {
  if (n_real <= 0) return cudaSuccess;
  rfe_fold_kernel<<<n_real, kThreads, 0, st>>>(tile_start, rs, partials, fac);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_rfe_apply(int n_tiles, cudaStream_t st, const RedTile* tiles, const RealDesc* rd,
                             const RowGeoD* geod, const RfeStep* rs, const double* fac, int phase, T* state) {
  if (n_tiles <= 0) return cudaSuccess;
  rfe_apply_kernel<T><<<n_tiles, kThreads, 0, st>>>(tiles, rd, geod, rs, fac, phase, state);
  return cudaGetLastError();
}

cudaError_t launch_fold(int mode, int n_real, cudaStream_t st, const int* tile_start,
                        const double* partials, const double* wpar, double* out) {
  if (n_real <= 0) return cudaSuccess;
  fold_kernel<<<n_real, kThreads, 0, st>>>(mode, tile_start, partials, wpar, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_apply(int mode, int n_tiles, cudaStream_t st, const RedTile* tiles,
                         const RealDesc* rd, const RowGeoD* geod, T* state, AssimArgs aa,
                         const double* factors) {
  if (n_tiles <= 0) return cudaSuccess;
  apply_kernel<T><<<n_tiles, kThreads, 0, st>>>(mode, tiles, rd, geod, state, aa, factors);
  return cudaGetLastError();
}

#define SFT_INSTANTIATE(T)                                                                       \
  template cudaError_t launch_rkl2_stage<T>(int, cudaStream_t, const Tile*, const RealDesc*,      \
                                            const StepParam*, const RowGeo<T>*, const ShapeConst*, \
                                            const Coef<T>*, T*, T*, T*, T*, int, int, int*);       \
  template cudaError_t launch_adv_stage<T>(int, cudaStream_t, const Tile*, const RealDesc*,       \
                                           const StepParam*, const RowGeo<T>*, const RowFlow<T>*, \
                                           const ShapeConst*, T*, T*, T*, AdvStage<T>);           \
  template cudaError_t launch_fix_poles<T>(int, cudaStream_t, const RealDesc*, T*, int);          \
  template cudaError_t launch_reduce<T>(int, int, cudaStream_t, const RedTile*, const RealDesc*,  \
                                        const RowGeoD*, const double*, const double*,             \
                                        const float4*, const T*, double, AssimArgs, double*);     \
  template cudaError_t launch_apply<T>(int, int, cudaStream_t, const RedTile*, const RealDesc*,   \
                                       const RowGeoD*, T*, AssimArgs, const double*);             \
  template cudaError_t launch_rfe_sums<T>(int, cudaStream_t, const RedTile*, const RealDesc*,     \
                                          const RowGeoD*, const RfeStep*, double*);              \
  template cudaError_t launch_rfe_apply<T>(int, cudaStream_t, const RedTile*, const RealDesc*,    \
                                           const RowGeoD*, const RfeStep*, const double*, int, T*);

SFT_INSTANTIATE(float)
SFT_INSTANTIATE(double)

}  // namespace sft
