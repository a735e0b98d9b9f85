/* ngf_cnn.h - tensor-core building blocks of a learned initializer for the
 * NGF registration of libngf_b300.
 *
 * A learned initializer maps a resampled image pair to a coarse deformation
 * that the Gauss-Newton method of Sec. 2.3 then refines from its first level
 * instead of from u = 0 (the multilevel start of Sec. 2.3 is left unchanged:
 * the network only supplies a different starting point).  Its dense work is
 * 3x3x3 convolution, which runs here as an implicit GEMM on the fifth
 * generation tensor cores (tcgen05.mma, BF16 operands, FP32 accumulation in
 * tensor memory).
 *
 * Layouts (all row-major, last index fastest):
 *   activations  x[B][D][H][W][Cin]        bf16, channels last
 *   weights      w[Cout][3][3][3][Cin]     bf16 (tap z, y, x, then channel)
 *   bias         b[Cout]                   float, may be NULL
 *   output       y[B][D][H][W][Cout]       float
 * The convolution is a cross-correlation with zero padding of one voxel and
 * stride 1 (output size = input size):
 *   y[n,z,y,x,o] = b[o] + sum_{dz,dy,dx in {-1,0,1}} sum_c
 *                  w[o, dz+1, dy+1, dx+1, c] * x[n, z+dz, y+dy, x+dx, c],
 * with x = 0 outside the volume; relu != 0 replaces negative outputs by 0.
 *
 * All pointers are device pointers owned by the caller, 16-byte aligned.
 * Constraints: Cin a multiple of 16 and (Cin <= 64 or a multiple of 64);
 * Cout a multiple of 16 in [16, 256]; B*D*H*W < 2^31; an empty volume is a
 * no-op.  Violations return NGF_EINVAL without launching.  The call is
 * asynchronous on `cuda_stream` (NULL = the legacy default stream).
 */
#ifndef NGF_CNN_H
#define NGF_CNN_H

#include "ngf.h"

#ifdef __cplusplus
extern "C" {
#endif

/* 3x3x3 convolution forward (see above).  The weights are first repacked
 * into a temporary of 27*Cout*Cin*2 bytes taken from the library's
 * stream-ordered pool (NGF_ENOMEM if that fails; released on the stream
 * after the launch); then one CTA computes an 8 x 16 x P block of output
 * voxels (P = 1, 2 or 4) for a slice of the output channels from an input
 * brick staged in shared memory once per 64 input channels.  Repeated calls
 * with the same arguments give identical results (no atomics; each output
 * accumulates (channel chunk, tap) in a fixed order). */
ngf_status ngf_conv3d_fwd(const void* x, const void* w, const float* bias, float* y,
                          int32_t B, int32_t D, int32_t H, int32_t W,
                          int32_t Cin, int32_t Cout, int32_t relu, void* cuda_stream);

/* Synchronises `cuda_stream` and returns the number of bounded waits of the
 * convolution kernels that gave up since the last call (0 in a healthy run;
 * a kernel that gives up leaves its output undefined but frees what it holds
 * and returns), or a negative ngf_status if the synchronisation failed. */
int32_t ngf_conv3d_check(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NGF_CNN_H */
