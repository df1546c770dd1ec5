// sfs_gemm.cuh -- the surrogate's training GEMM on the fifth-generation
// tensor cores: C = alpha op(A) op(B) + beta C + bias, BF16 operands, FP32
// accumulation in tensor memory (tcgen05.mma, M = 128), FP32 output.
//
// An operand is FP32 or BF16 in HBM, K-major (element (mn, k) at
// p[mn * ld + k]) or MN-major (at p[k * ld + mn]), with a batch stride
// (0: every batch shares it).  BF16 operands reach shared memory by TMA
// (cp.async.bulk.tensor, 128-byte swizzle); FP32 operands are rounded to
// BF16 (round to nearest even) by the threads that stage them into the same
// swizzled layout, so a product gives the same bits whichever way an
// operand is stored.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sfs_gemm {

enum DType : int { F32 = 0, BF16 = 1 };

struct Operand {
  const void* p;
  int dtype;      // F32 or BF16
  int mn_major;   // 0: p[mn*ld + k]; 1: p[k*ld + mn]
  long long ld;   // elements
  long long stride;  // elements between batches (0: shared)
};

struct Problem {
  int M, N, K;
  Operand a, b;
  float* C;
  long long ldc, sC;
  float alpha, beta;
  const float* bias;  // per column, may be null
  int kchunk;         // > 0: batch z covers k in [z*kchunk, (z+1)*kchunk) of one product (split-K)
  int batch;          // grid z extent (batches, or K chunks when kchunk > 0)
};

// Enqueue the product on `stream`.  `err` (device int) receives a nonzero
// code if a wait inside the kernel ran out of time (the kernel then returns
// without finishing its tile).  Returns the launch status; cudaErrorInvalidValue
// for arguments the kernel cannot take (a BF16 operand whose address, leading
// dimension or batch stride is not a multiple of 16 bytes).
cudaError_t launch(const Problem& pr, int* err, cudaStream_t stream);

// Shared-memory and attribute set-up of the kernels (idempotent).
cudaError_t prepare();

}  // namespace sfs_gemm
