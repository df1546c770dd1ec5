// sfs_fused.cuh -- internal interface of the fused inference forward pass of
// the surrogate (sfs_fused.cu), used by sfs.cu.  Not part of the C-ABI.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>

namespace sfs_fused {

constexpr int kChannels = 64;  // the configuration the fused kernel is written for
constexpr int kModes = 48;
constexpr int kMaxBlocks = 4;

// Offsets (in floats) of the FP32 master parameters (the order of sfs.h).
struct ParamOffsets {
  long long We, be, Wd, bd;
  long long w[kMaxBlocks], W1[kMaxBlocks], b1[kMaxBlocks], W2[kMaxBlocks], b2[kMaxBlocks];
};

// Bytes of the BF16 weight image (the shared-memory layout the kernel
// copies) and of the kernel's dynamic shared memory, for L blocks.
size_t image_bytes(int L);
size_t smem_bytes(int L);

// Raise the kernel's dynamic shared-memory limit (once per process).
cudaError_t prepare(int L);

// Build the image from the FP32 master parameters P and the latent DFT
// matrices Fm [96][128], Gm [128][96] (FP32 device arrays).
cudaError_t build_image(const float* P, const ParamOffsets& o, int L, const float* Fm, const float* Gm,
                        unsigned char* img, cudaStream_t st);

// delta[b][row][col] (unpatched decoder output, before the centring) of nb
// maps from x, the rotated maps r, the parameters p[nb][5] and the spectral
// weights in P; one persistent block per SM (grid = min(n_sm, nb * 64)).
cudaError_t forward(const unsigned char* img, int L, const float* P, const ParamOffsets& o, const float* x,
                    const float* r, const float* p, int nb, float* delta, int n_sm, cudaStream_t st);

}  // namespace sfs_fused
