/*
 * sfs.h -- C-ABI of the learned one-day surrogate of libsft (GB300, sm_103a).
 *
 * The paper has no learned component (its introduction only mentions a
 * PINN-based SFT); this network proposes one-day advances of 256 x 512 maps
 * for ensemble members, with the plain solver of sft.h as judge and fallback.
 *
 * Network (per map x [256][512] in Gauss, parameters p[5] = Omega
 * coefficients o0, o2, o4 in deg/day, meridional amplitude U in m/s,
 * diffusivity eta in km^2/s):
 *   r      = x rotated per row in phi by the day's differential rotation
 *            (Omega(lat) - 360/27.2753 deg/day, exact in phi-Fourier space)
 *   h      = 4x4-strided patch embedding of [x, r]/100 G, p, cos/sin(colat)
 *   blocks = L x { per-latent-row phi-spectral mixing (M modes, complex
 *            weights per row/mode/channel) + residual;
 *            channel MLP C -> 2C -> C with GELU + residual }
 *   x_next = r + 100 G * unpatchify(h Wd + bd)
 * Every learned contraction is a BF16 tensor-core product with FP32
 * accumulation: in training a tcgen05 GEMM (accumulator in tensor memory;
 * BF16 activations by TMA, FP32 ones rounded to BF16 as they are staged), in
 * inference one fused mma.sync kernel; the fixed rotation is an FP32 FFT per
 * map row (the 512-point DFT, the phase, the inverse transform).  Master
 * weights, gradients and AdamW moments are FP32.
 *
 * Parameter vector order (FP32, flat): We[48][C], be[C], Wd[C][16], bd[16],
 * then per block l: w_l[64][M][C][2], W1_l[C][2C], b1_l[2C], W2_l[2C][C],
 * b2_l[C].
 *
 * All map/parameter pointers are device pointers (FP32, row-major) of the
 * current device, maps 16-byte aligned (SFT_ERR_ARG otherwise); work is queued on the handle's stream; errors are status
 * codes with text in sft_last_error(NULL).
 */
#ifndef SFS_H_
#define SFS_H_

#include <stdint.h>

#include "sft.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sfs_net* sfs_handle;

typedef struct {
  int32_t channels;   /* C, multiple of 16 */
  int32_t modes;      /* M spectral modes kept (<= 64) */
  int32_t blocks;     /* L */
  int32_t max_batch;  /* largest batch passed to forward / train */
  uint64_t seed;      /* weight initialisation */
} sfs_config;

/* Create a network (weights initialised from seed) and its work buffers for
 * batches up to max_batch.  cuda_stream as in sft_create_grid. */
sft_status sfs_create(const sfs_config* cfg, void* cuda_stream, sfs_handle* out);

/* Frees the network and its buffers after the work queued on its stream. */
sft_status sfs_destroy(sfs_handle h);

/* Number of FP32 parameters. */
int64_t sfs_num_params(sfs_handle h);

/* Copy the flat parameter vector in / out (host arrays of sfs_num_params). */
sft_status sfs_set_params(sfs_handle h, const float* host_params);

/* The current flat parameter vector, copied out to host_params. */
sft_status sfs_get_params(sfs_handle h, float* host_params);

/* y[b] = surrogate one-day advance of x[b] with parameters p[b] (device
 * arrays x, y [n][256][512], p [n][5]); n <= max_batch. */
sft_status sfs_forward(sfs_handle h, const float* x, const float* p, int32_t n, float* y);

/* Loss mean_b ||x_next - y||^2/||y||^2 and its gradient for the current
 * weights (host arrays: *loss, grad[sfs_num_params]).  Synchronises. */
sft_status sfs_loss_grad(sfs_handle h, const float* x, const float* p, const float* y, int32_t n,
                         float* loss, float* host_grad);

/* One AdamW step (beta1 0.9, beta2 0.999, eps 1e-8, decoupled weight
 * decay wd) on the loss above.  *loss (host, may be NULL) receives the loss
 * of this batch before the update (synchronises when not NULL). */
sft_status sfs_train_step(sfs_handle h, const float* x, const float* p, const float* y, int32_t n,
                          double lr, double wd, float* loss);

/* Relative L2 error ||a_b - b_b|| / ||b_b|| of n maps (device) into host out[n] (FP64
 * accumulation).  Any n >= 1 (reduced max_batch maps at a time); synchronises
 * once. */
sft_status sfs_rel_l2(sfs_handle h, const float* a, const float* b, int32_t n, double* out);

/* Total flux sum A B and unsigned flux sum A |B| (code units, FP64) of n
 * maps (device [n][256][512]) into host out[2n], with the grid convention of
 * sft.h (poles included, caps of area 2 pi (1 - cos(dtheta/2))); the judge
 * of the surrogate ensemble uses them for the flux-drift test.  Any n >= 1
 * (reduced max_batch maps at a time); synchronises once. */
sft_status sfs_flux(sfs_handle h, const float* maps, int32_t n, double* out);

/* SMs the fused inference forward may occupy (its persistent blocks hold
 * most of an SM's shared memory each); 0 (the default) means all.  A caller
 * that runs solver work on another stream beside the forward passes leaves
 * the remaining SMs to it.  No counterpart in the paper (a scheduling
 * control of this implementation). */
sft_status sfs_set_sm_budget(sfs_handle h, int32_t n_sm);

/* One training-pass product on the handle's stream, for tests of the tensor-
 * core GEMM: C[z] = alpha A[z] B[z] + beta C[z] + bias (A: M x K, B: K x N,
 * device pointers).  Operand element (mn, k) is at p[mn*ld + k] (mn_major 0)
 * or p[k*ld + mn] (mn_major 1), batch z at p + z*stride (stride 0: shared);
 * *_bf16 = 1 for BF16 operands (16-byte aligned, ld and stride multiples of
 * 8), 0 for FP32 (rounded to BF16, nearest even, as staged).  C is FP32,
 * C[z][m*ldc + n] with C + z*sC; bias (may be NULL) is per column.  kchunk > 0
 * splits K into batch chunks of kchunk (partial products into C[z], the
 * operands unbatched).  Synchronises; SFT_ERR_CUDA if a wait inside the
 * kernel ran out of time.  No counterpart in the paper (a test entry point). */
sft_status sfs_debug_gemm(sfs_handle h, int32_t M, int32_t N, int32_t K, const void* A, int32_t a_bf16,
                          int32_t a_mn_major, int64_t lda, int64_t sA, const void* B, int32_t b_bf16,
                          int32_t b_mn_major, int64_t ldb, int64_t sB, float* C, int64_t ldc, int64_t sC,
                          float alpha, float beta, const float* bias, int32_t kchunk, int32_t batch);

/* Counters: GEMM launches and floating-point operations issued so far. */
sft_status sfs_counters(sfs_handle h, int64_t* gemm_launches, double* gemm_flops, int64_t* kernel_launches);

#ifdef __cplusplus
}
#endif

#endif /* SFS_H_ */
