// sfs_gemm.cu -- tcgen05 GEMM of the surrogate's training pass (sfs_gemm.cuh).
//
// A persistent CTA of 256 threads computes 128 x BN tiles of C (BN = 64 or
// 128) in 64-wide K steps:
//  * operand tiles live in shared memory as 128-byte swizzled atoms
//    (8 rows of 128 bytes, 16-byte chunks XOR-ed with the row), K-major
//    (row = mn, 64 k per row) or MN-major (row = k, 64 mn per row), in a
//    ring of NST stages;
//  * BF16 operands are copied by TMA (one box per operand and stage for a
//    K-major tile, one per 64 mn for an MN-major tile), completing on the
//    stage's `full` mbarrier;
//  * FP32 operands are loaded a stage ahead into registers by all threads,
//    rounded to BF16 and stored into the swizzled layout;
//  * thread 0 issues tcgen05.mma (kind::f16, BF16 x BF16 -> FP32, M = 128,
//    N = BN, K = 16 each) on the stage and commits it to the stage's `done`
//    mbarrier, which frees the stage for the next load;
//  * the accumulator is BN columns of tensor memory; the epilogue reads it
//    with tcgen05.ld (warp w: lanes 32 (w mod 4) .. +31, half w / 4 of the
//    columns), transposes each warp's 32 x 32 block through padded shared
//    memory and writes rows of 128 contiguous bytes, with alpha, beta and
//    bias applied;
//  * a CTA takes output tiles in turn (two CTAs per SM); the next tile's
//    first operands are loaded and copied while the current accumulator is
//    read out.
// Every mbarrier wait gives up after about two seconds of global time: the
// kernel then records a code in *err, waits (again bounded) for the copies
// and products it issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "sfs_gemm.cuh"

namespace sfs_gemm {
namespace {

constexpr int BM = 128, BK = 64, THREADS = 256;
constexpr int ATOM = 1024;                // 8 rows x 128 bytes
constexpr int A_BYTES = BM * BK * 2;      // 16 KB
constexpr unsigned long long kWaitNs = 2000000000ull;

constexpr int SCR_FLOATS = 32 * 33;  // a warp's 32 x 32 output block, rows padded to 33 floats

template <int BN>
struct Cfg {
  static constexpr int B_BYTES = BN * BK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int NST = BN == 128 ? 2 : 3;  // two CTAs per SM either way
  static constexpr int TMEM_COLS = BN;           // power of two >= 32
  // alignment slack, the stages (1024-aligned), the epilogue's transpose
  // scratch (8 warps), 2 NST mbarriers and the TMEM address
  static constexpr int SCRATCH = (THREADS / 32) * SCR_FLOATS * 4;
  static constexpr int SMEM = 1024 + NST * STAGE + SCRATCH + 2 * NST * 8 + 16;
};

struct OpDev {
  const char* p;
  long long ld, stride;  // elements
  int dtype, mn, tma, vec;
};

struct Args {
  int M, N, K;
  OpDev a, b;
  float* C;
  long long ldc, sC;
  float alpha, beta;
  const float* bias;
  int kchunk, nz;
  int* err;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase of parity `par` has completed; false after kWaitNs
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t par) {
  const unsigned long long t0 = global_ns();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(par)
        : "memory");
    if (ok) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void record_error(int* err, int code) {
  if (err) atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap* map, int x, int y, int z, int rank,
                                         uint32_t bar) {
  const uint64_t m = reinterpret_cast<uint64_t>(map);
  if (rank == 3)
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"(m), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
  else
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(m), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------- tcgen05
// Shared-memory matrix descriptor, 128-byte swizzle: start address, leading
// and stride byte offsets (>> 4), fixed version 1 at bit 46, swizzle mode 2
// at bits 61..63.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A
// and B BF16 (bits 7-9, 10-12 = 1), A/B MN-major flags (bits 15, 16), N >> 3
// (bits 17-22), M >> 4 (bits 24-28).
__host__ __device__ constexpr uint32_t idesc(int n, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- staging
// Byte offset of element (r, k) in a K-major tile (row r = mn, 64 k per row)
// and in an MN-major tile (row = k, 64 mn per row; atoms of 64 mn are 8192
// bytes apart).  The XOR of the 16-byte chunk with the row within its
// 8-row atom is the 128-byte swizzle that TMA writes and tcgen05 reads.
__device__ __forceinline__ uint32_t off_k(int r, int k) {
  return (uint32_t)((r >> 3) * ATOM + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) << 4) | ((k & 7) << 1)));
}
__device__ __forceinline__ uint32_t off_mn(int r, int k) {
  return (uint32_t)((r >> 6) * (8 * ATOM) + (k >> 3) * ATOM + (k & 7) * 128 +
                    (((((r & 63) >> 3) ^ (k & 7)) << 4) | ((r & 7) << 1)));
}

// Group i of this thread in an R x 64 tile: 4 consecutive elements along
// the operand's contiguous dimension.
template <int R>
__device__ __forceinline__ void group_coords(int mn, int i, int& r, int& k) {
  const int g = (int)threadIdx.x + THREADS * i;
  if (!mn) { r = g >> 4; k = (g & 15) << 2; }
  else { k = g / (R / 4); r = (g % (R / 4)) << 2; }
}

__device__ __forceinline__ float ld_f(const char* p, long long e) { return reinterpret_cast<const float*>(p)[e]; }

// Global -> registers (FP32 operands): R/16 groups of 4 floats, zeros
// outside [0, mn_end) x [k0, k_end).
template <int R>
__device__ __forceinline__ void load_groups(const OpDev& o, const char* base, int mn0, int k0, int mn_end, int k_end,
                                            uint4 (&v)[R / 16]) {
#pragma unroll
  for (int i = 0; i < R / 16; ++i) {
    int r, k;
    group_coords<R>(o.mn, i, r, k);
    const int gr = mn0 + r, gk = k0 + k;
    float f[4] = {0.f, 0.f, 0.f, 0.f};
    if (!o.mn) {
      if (gr < mn_end) {
        const long long e0 = (long long)gr * o.ld + gk;
        if (o.vec && gk + 3 < k_end) {
          const float4 t = *reinterpret_cast<const float4*>(base + 4 * e0);
          f[0] = t.x; f[1] = t.y; f[2] = t.z; f[3] = t.w;
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) if (gk + e < k_end) f[e] = ld_f(base, e0 + e);
        }
      }
    } else if (gk < k_end) {
      const long long e0 = (long long)gk * o.ld + gr;
      if (o.vec && gr + 3 < mn_end) {
        const float4 t = *reinterpret_cast<const float4*>(base + 4 * e0);
        f[0] = t.x; f[1] = t.y; f[2] = t.z; f[3] = t.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) if (gr + e < mn_end) f[e] = ld_f(base, e0 + e);
      }
    }
    const uint4 x = make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), __float_as_uint(f[3]));
    v[i] = x;
  }
}

// Registers -> the stage's swizzled tile (FP32 rounded to BF16, nearest even).
template <int R>
__device__ __forceinline__ void store_groups(const OpDev& o, uint8_t* tile, const uint4 (&v)[R / 16]) {
#pragma unroll
  for (int i = 0; i < R / 16; ++i) {
    int r, k;
    group_coords<R>(o.mn, i, r, k);
    const __nv_bfloat162 lo = __floats2bfloat162_rn(__uint_as_float(v[i].x), __uint_as_float(v[i].y));
    const __nv_bfloat162 hi = __floats2bfloat162_rn(__uint_as_float(v[i].z), __uint_as_float(v[i].w));
    uint2 w;
    w.x = *reinterpret_cast<const uint32_t*>(&lo);
    w.y = *reinterpret_cast<const uint32_t*>(&hi);
    *reinterpret_cast<uint2*>(tile + (o.mn ? off_mn(r, k) : off_k(r, k))) = w;
  }
}

// Descriptor of k-step j (16 k) of a tile.  K-major: the step is 32 bytes
// along the swizzled row; the stride offset (next 8 rows) is one atom.
// MN-major: the step is two 8-row k groups; the leading offset steps to
// the next 64 mn, the stride offset to the next 8 k.
#ifndef SFS_MN_LBO
#define SFS_MN_LBO (8 * ATOM)
#define SFS_MN_SBO ATOM
#endif
__device__ __forceinline__ uint64_t tile_desc(uint32_t tile, int mn, int j) {
  return mn ? sdesc(tile + (uint32_t)j * 2 * ATOM, SFS_MN_LBO, SFS_MN_SBO) : sdesc(tile + (uint32_t)j * 32, 16, ATOM);
}

// TMA of one operand tile into `dst`: K-major, one box of 64 k x R rows;
// MN-major, R/64 boxes of 64 mn x 64 k.
template <int R>
__device__ __forceinline__ void tma_tile(const CUtensorMap* map, int rank, int mn_major, uint32_t dst, int mn0, int k0,
                                         int z, uint32_t bar) {
  if (!mn_major) {
    tma_load(dst, map, k0, mn0, z, rank, bar);
  } else {
#pragma unroll
    for (int q = 0; q < R / 64; ++q) tma_load(dst + q * 8 * ATOM, map, mn0 + 64 * q, k0, z, rank, bar);
  }
}

__device__ __forceinline__ int esize(int dtype) { return dtype == F32 ? 4 : 2; }

// ---------------------------------------------------------------- kernel
// The output tiles (x: N tile, y: M tile, z: batch or K chunk) are numbered
// t = (z ny + y) nx + x; CTA b takes t = b, b + gridDim.x, ... (persistent).
// The k tiles of all its output tiles share one count gk: k tile gk uses
// stage gk mod NST and completes phase gk / NST of that stage's barriers.
// The next output tile's first operands are loaded (registers) and copied
// (TMA) while the current tile's accumulator is read out.
struct Tile {
  int n0, m0, z, kb0, kb1, nk, za, zb;
  const char *pa, *pb;
};

template <int BN>
__global__ void __launch_bounds__(THREADS, 2)
    gemm_tc_kernel(const Args g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   int rankA, int rankB) {
  using CF = Cfg<BN>;
  constexpr int NST = CF::NST;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  float* scratch = reinterpret_cast<float*>(sm + NST * CF::STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + NST * CF::STAGE + CF::SCRATCH);  // full[NST], done[NST]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NST);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nx = (g.N + BN - 1) / BN, ny = (g.M + BM - 1) / BM;
  const long long ntiles = (long long)nx * ny * g.nz;
  const bool split = g.kchunk > 0;
  const uint32_t full0 = smem_u32(bars), done0 = smem_u32(bars + NST);
  const uint32_t st0 = smem_u32(sm);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(CF::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int s = 0; s < 2 * NST; ++s) bar_init(full0 + 8 * s, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  const bool reg_a = !g.a.tma, reg_b = !g.b.tma, any_tma = g.a.tma || g.b.tma;
  const uint32_t tx = (g.a.tma ? A_BYTES : 0) + (g.b.tma ? CF::B_BYTES : 0);
  const uint32_t id = idesc(BN, g.a.mn, g.b.mn);
  auto tile_of = [&](long long t, Tile& ti) {
    const int x = (int)(t % nx);
    const long long r = t / nx;
    ti.n0 = x * BN;
    ti.m0 = (int)(r % ny) * BM;
    ti.z = (int)(r / ny);
    ti.kb0 = split ? ti.z * g.kchunk : 0;
    ti.kb1 = split ? min(g.K, ti.kb0 + g.kchunk) : g.K;
    ti.nk = ti.kb1 > ti.kb0 ? (ti.kb1 - ti.kb0 + BK - 1) / BK : 0;
    const int zo = split ? 0 : ti.z;  // operand batch
    ti.pa = g.a.p + (long long)zo * g.a.stride * esize(g.a.dtype);
    ti.pb = g.b.p + (long long)zo * g.b.stride * esize(g.b.dtype);
    ti.za = rankA == 3 ? zo : 0;
    ti.zb = rankB == 3 ? zo : 0;
  };
  auto issue_tma = [&](const Tile& ti, int kt, uint32_t gi) {  // thread 0: the TMA part of k tile kt
    const int s = (int)(gi % NST), k = ti.kb0 + kt * BK;
    const uint32_t bar = full0 + 8 * s, sa = st0 + s * CF::STAGE;
    bar_expect_tx(bar, tx);
    if (g.a.tma) tma_tile<BM>(&tmA, rankA, g.a.mn, sa, ti.m0, k, ti.za, bar);
    if (g.b.tma) tma_tile<BN>(&tmB, rankB, g.b.mn, sa + A_BYTES, ti.n0, k, ti.zb, bar);
  };
  auto load_regs = [&](const Tile& ti, int kt, uint4 (&ra)[BM / 16], uint4 (&rb)[BN / 16]) {
    const int k = ti.kb0 + kt * BK;
    if (reg_a) load_groups<BM>(g.a, ti.pa, ti.m0, k, g.M, ti.kb1, ra);
    if (reg_b) load_groups<BN>(g.b, ti.pb, ti.n0, k, g.N, ti.kb1, rb);
  };

  uint4 ra[BM / 16], rb[BN / 16];
  long long t = blockIdx.x;
  Tile cur{};
  uint32_t gk = 0;     // k tiles of the previous output tiles
  int tma_next = 0;    // thread 0: k tiles of `cur` whose TMA was issued
  int committed = -1;  // thread 0: last k tile of `cur` whose products were committed
  bool bad = false;
  if (t < ntiles) {
    tile_of(t, cur);
    if (cur.nk > 0) load_regs(cur, 0, ra, rb);
    if (tid == 0 && any_tma)
      for (; tma_next < min(NST, cur.nk); ++tma_next) issue_tma(cur, tma_next, gk + tma_next);
  }
  for (; t < ntiles; t += gridDim.x) {
    Tile nxt{};
    const bool has_next = t + gridDim.x < ntiles;
    if (has_next) tile_of(t + gridDim.x, nxt);
    committed = -1;
    for (int kt = 0; kt < cur.nk; ++kt) {
      const uint32_t gi = gk + kt;
      const int s = (int)(gi % NST);
      uint8_t* sa = sm + s * CF::STAGE;
      if (reg_a || reg_b) {
        // the stage is free once the products of k tile gi - NST completed
        if (gi >= NST && !bar_wait(done0 + 8 * s, ((gi / NST) - 1) & 1)) bad = true;
        if (!bad) {
          if (reg_a) store_groups<BM>(g.a, sa, ra);
          if (reg_b) store_groups<BN>(g.b, sa + A_BYTES, rb);
          fence_async_smem();
        }
        if (kt + 1 < cur.nk) load_regs(cur, kt + 1, ra, rb);
        else if (has_next && nxt.nk > 0) load_regs(nxt, 0, ra, rb);
      }
      if (__syncthreads_or(bad)) {
        bad = true;
        break;
      }
      if (tid == 0) {
        if (any_tma && !bar_wait(full0 + 8 * s, (gi / NST) & 1)) {
          bad = true;
        } else {
          fence_after_sync();
          const uint32_t sa32 = st0 + s * CF::STAGE, sb32 = sa32 + A_BYTES;
          const int nmma = (min(BK, cur.kb1 - (cur.kb0 + kt * BK)) + 15) / 16;
          for (int j = 0; j < nmma; ++j)
            mma_bf16(tmem, tile_desc(sa32, g.a.mn, j), tile_desc(sb32, g.b.mn, j), id, (kt > 0 || j > 0) ? 1u : 0u);
          mma_commit(done0 + 8 * s);
          committed = kt;
          // refill the stage of k tile kt - 1 (its products have had a step to finish)
          if (any_tma && kt >= 1 && tma_next < cur.nk) {
            const uint32_t gp = gi - 1;
            if (!bar_wait(done0 + 8 * (gp % NST), (gp / NST) & 1)) bad = true;
            else { issue_tma(cur, tma_next, gk + tma_next); ++tma_next; }
          }
        }
      }
    }
    if (!bad && cur.nk > 0) {
      const uint32_t gl = gk + cur.nk - 1;
      if (!bar_wait(done0 + 8 * (gl % NST), (gl / NST) & 1)) bad = true;
    }
    bad = __syncthreads_or(bad);
    if (bad) break;
    // every stage is free: start the next tile's copies before the read-out
    const uint32_t gn = gk + cur.nk;
    if (tid == 0) {
      tma_next = 0;
      if (any_tma && has_next)
        for (; tma_next < min(NST, nxt.nk); ++tma_next) issue_tma(nxt, tma_next, gn + tma_next);
    }
    fence_after_sync();
    {
      // warp w reads lanes 32 (w mod 4) .. +31 (rows) of column half w / 4
      // in 32 x 32 blocks, transposes each through its padded scratch and
      // writes it row by row: lane = column, 128 contiguous bytes a store
      const int q = warp & 3, h = warp >> 2;
      float* scr = scratch + warp * SCR_FLOATS;
      float* C = g.C + (long long)cur.z * g.sC;
#pragma unroll
      for (int c = 0; c < BN / 2; c += 32) {
        float v[32];
        if (cur.nk > 0) {
          tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * (BN / 2) + c), v);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) scr[lane * 33 + i] = v[i];
        __syncwarp();
        const int col = cur.n0 + h * (BN / 2) + c + lane;
        const bool cok = col < g.N;
        const float bv = (g.bias && cok) ? g.bias[col] : 0.f;
        const int r0 = cur.m0 + 32 * q;
        const int nr = min(32, g.M - r0);
        float* cp = C + (long long)r0 * g.ldc + col;
        if (cok) {
          if (g.beta != 0.f) {
            for (int r8 = 0; r8 < nr; r8 += 8) {  // eight reads of C in flight before their writes
              float cv[8];
#pragma unroll
              for (int r = 0; r < 8; ++r) cv[r] = r8 + r < nr ? cp[(long long)(r8 + r) * g.ldc] : 0.f;
#pragma unroll
              for (int r = 0; r < 8; ++r)
                if (r8 + r < nr)
                  cp[(long long)(r8 + r) * g.ldc] = g.alpha * scr[(r8 + r) * 33 + lane] + g.beta * cv[r] + bv;
            }
          } else {
#pragma unroll 8
            for (int r = 0; r < nr; ++r) cp[(long long)r * g.ldc] = g.alpha * scr[r * 33 + lane] + bv;
          }
        }
        __syncwarp();
      }
    }
    fence_before_sync();  // the next tile's products overwrite the accumulator after its first barrier
    gk = gn;
    cur = nxt;
  }
  if (bad && tid == 0) {
    record_error(g.err, 1);
    // bounded waits for what this CTA still has in flight
    if (committed >= 0) {
      const uint32_t gc = gk + committed;
      bar_wait(done0 + 8 * (gc % NST), (gc / NST) & 1);
    }
    for (int kt = committed + 1; kt < tma_next; ++kt) {
      const uint32_t gt = gk + kt;
      bar_wait(full0 + 8 * (gt % NST), (gt / NST) & 1);
    }
  }
  fence_before_sync();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CF::TMEM_COLS) : "memory");
}

}  // namespace

// ---------------------------------------------------------------- host
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// TMA needs a 16-byte aligned base, leading dimension and batch stride.
bool tma_ok(const Operand& o) {
  if (o.dtype != BF16) return false;
  const long long es = 2;
  return (reinterpret_cast<uintptr_t>(o.p) & 15) == 0 && (o.ld * es) % 16 == 0 && (o.stride * es) % 16 == 0;
}

bool vec_ok(const Operand& o) {
  const int es = o.dtype == F32 ? 4 : 2;
  return (reinterpret_cast<uintptr_t>(o.p) % (4 * es)) == 0 && o.ld % 4 == 0 && o.stride % 4 == 0;
}

// Tensor map of a BF16 operand with `rows` mn and K extent, batched when
// rank == 3: K-major boxes are 64 k x box_rows, MN-major boxes 64 mn x 64 k.
cudaError_t make_map(CUtensorMap* map, const Operand& o, int rows, int K, int batch, int rank, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  cuuint64_t dims[3], strides[2];
  cuuint32_t box[3], estr[3] = {1, 1, 1};
  if (!o.mn_major) {
    dims[0] = (cuuint64_t)K; dims[1] = (cuuint64_t)rows;
    box[0] = BK; box[1] = (cuuint32_t)box_rows;
  } else {
    dims[0] = (cuuint64_t)rows; dims[1] = (cuuint64_t)K;
    box[0] = 64; box[1] = BK;
  }
  dims[2] = (cuuint64_t)batch;
  box[2] = 1;
  strides[0] = (cuuint64_t)(o.ld * 2);
  strides[1] = (cuuint64_t)(o.stride * 2);
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void*>(o.p), dims, strides,
                        box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// CTAs of the BN kernel resident on the whole GPU (set by prepare)
int g_resident[2] = {0, 0};
int g_occ[2] = {0, 0};
template <int BN>
int resident() { return g_resident[BN == 128 ? 1 : 0]; }

template <int BN>
cudaError_t launch_bn(const Problem& pr, int* err, cudaStream_t stream) {
  const bool split = pr.kchunk > 0;
  Args g{};
  g.M = pr.M; g.N = pr.N; g.K = pr.K;
  g.C = pr.C; g.ldc = pr.ldc; g.sC = pr.sC;
  g.alpha = pr.alpha; g.beta = pr.beta; g.bias = pr.bias;
  g.kchunk = pr.kchunk;
  g.err = err;
  CUtensorMap maps[2];
  int ranks[2] = {2, 2};
  const Operand* ops[2] = {&pr.a, &pr.b};
  OpDev* devs[2] = {&g.a, &g.b};
  for (int i = 0; i < 2; ++i) {
    const Operand& o = *ops[i];
    OpDev& d = *devs[i];
    d.p = static_cast<const char*>(o.p);
    d.ld = o.ld; d.stride = o.stride; d.dtype = o.dtype; d.mn = o.mn_major;
    d.vec = vec_ok(o) ? 1 : 0;
    d.tma = tma_ok(o) ? 1 : 0;
    memset(&maps[i], 0, sizeof(CUtensorMap));
    if (d.tma) {
      const int rows = i == 0 ? pr.M : pr.N;
      ranks[i] = (!split && pr.batch > 1 && o.stride != 0) ? 3 : 2;
      const cudaError_t e = make_map(&maps[i], o, rows, pr.K, ranks[i] == 3 ? pr.batch : 1, ranks[i], i == 0 ? BM : BN);
      if (e != cudaSuccess) return e;
    } else if (o.dtype == BF16) {
      return cudaErrorInvalidValue;  // a BF16 operand TMA cannot address
    }
  }
  g.nz = pr.batch;
  const long long ntiles = (long long)((pr.N + BN - 1) / BN) * ((pr.M + BM - 1) / BM) * pr.batch;
  const int grid = (int)std::min<long long>(ntiles, (long long)resident<BN>());
  gemm_tc_kernel<BN><<<grid, THREADS, Cfg<BN>::SMEM, stream>>>(g, maps[0], maps[1], ranks[0], ranks[1]);
  return cudaGetLastError();
}

}  // namespace

cudaError_t prepare() {
  static cudaError_t st = cudaErrorNotReady;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, sms = 0, smem_sm = 0, b64 = 0, b128 = 0;
    st = cudaGetDevice(&dev);
    if (st == cudaSuccess) st = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (st == cudaSuccess) st = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(gemm_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<64>::SMEM);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(gemm_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<128>::SMEM);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(gemm_tc_kernel<64>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
    if (st == cudaSuccess)
      st = cudaFuncSetAttribute(gemm_tc_kernel<128>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
    if (st == cudaSuccess)
      st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b64, gemm_tc_kernel<64>, THREADS, Cfg<64>::SMEM);
    if (st == cudaSuccess)
      st = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b128, gemm_tc_kernel<128>, THREADS, Cfg<128>::SMEM);
    g_occ[0] = b64;
    g_occ[1] = b128;
    // CTAs per SM: the launch bounds (2), the SM's shared memory (1 KB of
    // it reserved per CTA) and its tensor memory (512 columns)
    auto per_sm = [&](int smem, int cols, int api) {
      const int by_smem = smem_sm / (smem + 1024);
      return std::max(1, std::max(api, std::min(2, std::min(by_smem, 512 / cols))));
    };
    g_resident[0] = sms * per_sm(Cfg<64>::SMEM, 64, b64);
    g_resident[1] = sms * per_sm(Cfg<128>::SMEM, 128, b128);
  });
  return st;
}

cudaError_t launch(const Problem& pr, int* err, cudaStream_t stream) {
  if (pr.M <= 0 || pr.N <= 0 || pr.K < 0 || pr.batch <= 0 || !pr.C || !pr.a.p || !pr.b.p) return cudaErrorInvalidValue;
  const cudaError_t e = prepare();
  if (e != cudaSuccess) return e;
  return pr.N > 64 ? launch_bn<128>(pr, err, stream) : launch_bn<64>(pr, err, stream);
}

}  // namespace sfs_gemm
