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
 * brick copied to shared memory (TMA) once per 64 input channels; slices of
 * at most 64 output channels multiply the three z taps of a (dy, dx) in one
 * MMA.  Repeated calls with the same arguments give identical results (no
 * atomics; each output accumulates its products in a fixed order). */
ngf_status ngf_conv3d_fwd(const void* x, const void* w, const float* bias, float* y,
                          int32_t B, int32_t D, int32_t H, int32_t W,
                          int32_t Cin, int32_t Cout, int32_t relu, void* cuda_stream);

/* Flags of the convolution calls below. */
enum { NGF_CONV_RELU = 1,      /* replace negative outputs by 0                 */
       NGF_CONV_OUT_BF16 = 2   /* write the output as bf16 instead of float     */
};

/* As ngf_conv3d_fwd with flags (NGF_CONV_RELU, NGF_CONV_OUT_BF16): y is
 * float [B][D][H][W][Cout], or bf16 (round to nearest even) with
 * NGF_CONV_OUT_BF16; other flag bits return NGF_EINVAL. */
ngf_status ngf_conv3d_fwd_ex(const void* x, const void* w, const float* bias, void* y,
                             int32_t B, int32_t D, int32_t H, int32_t W,
                             int32_t Cin, int32_t Cout, int32_t flags, void* cuda_stream);

/* Data gradient of the convolution y = conv(x, w) of a layer with Cin input
 * and Cout output channels (the transpose of the forward map in x):
 *   dx[n,z,y,x,c] = sum_{taps, o} w[o, tap, c] * dy[n, (z,y,x) - tap, o],
 * dy [B][D][H][W][Cout] bf16, w [Cout][3][3][3][Cin] bf16 (the layer's own
 * weights), dx [B][D][H][W][Cin] float, or bf16 with NGF_CONV_OUT_BF16.  It
 * runs as the forward kernel on the mirrored taps with the channel roles
 * swapped, so Cout must satisfy the forward's Cin rule (a multiple of 16,
 * <= 64 or a multiple of 64) and Cin its Cout rule (16 .. 256, multiple of
 * 16).  FP32 accumulation; deterministic. */
ngf_status ngf_conv3d_dgrad(const void* dy, const void* w, void* dx,
                            int32_t B, int32_t D, int32_t H, int32_t W,
                            int32_t Cin, int32_t Cout, int32_t flags, void* cuda_stream);

/* Weight and bias gradients of the same layer:
 *   dw[o, tap, c] = sum_{n,z,y,x} dy[n,z,y,x,o] * x[n, (z,y,x) + tap, c]
 *   db[o]         = sum_{n,z,y,x} dy[n,z,y,x,o]
 * dy bf16 [..][Cout], x bf16 [..][Cin], dw float [Cout][3][3][3][Cin]
 * (overwritten), db float [Cout] or NULL.  The weight gradient is an
 * implicit GEMM on the tensor cores (rows: output channels, columns: input
 * channels, reduction: voxels, one tensor-memory accumulator per tap),
 * summed over the thread blocks in a fixed order; partial sums live in a
 * temporary from the library's stream-ordered pool.  Cin as for the forward,
 * Cout a multiple of 16 in [16, 128].  Deterministic. */
ngf_status ngf_conv3d_wgrad(const void* dy, const void* x, float* dw, float* db,
                            int32_t B, int32_t D, int32_t H, int32_t W,
                            int32_t Cin, int32_t Cout, void* cuda_stream);

/* ---- the learned initializer: a 3-D encoder-decoder ----------------------
 * Maps an image pair (R, T) of s^3 voxels (s a multiple of 8) to a
 * displacement on the (s/4 + 1)^3 node grid of the registration level with
 * s/2 image cells per axis and two image cells per deformation cell, from
 * which the multilevel Gauss-Newton method (Sec. 2.3) then continues
 * (register_multilevel's u_init / start_level).  The paper has no network:
 * it starts from u = 0 on the coarsest level; this only supplies another
 * start.  Layers (bf16 activations, FP32 accumulation, channels last):
 *   x0 = [(R - in_shift) in_scale, (T - in_shift) in_scale, 0 x 14]   s^3
 *   e1 = relu(conv W1) 16 ch, s^3;  p1 = mean-pool 2
 *   e2 = relu(conv W2) 32 ch, s/2;  p2 = mean-pool 2
 *   e3 = relu(conv W3) 64 ch, s/4;  p3 = mean-pool 2
 *   e4 = relu(conv W4) 128 ch, s/8
 *   d3 = relu(conv W5 of nearest-upsampled e4) 64 ch, s/4;  s3 = d3 + e3
 *   d2 = relu(conv W6 of s3) 64 ch;  o = conv W7 of d2 (16 ch, float)
 *   u  = out_scale * cell_to_node(o[..., 0:3]): node k of an axis is the mean
 *        of cells k-1 and k (clamped to the grid), component-major 3 x Nn
 *   loss = mean over pairs, components and nodes of ((u - u_target)/out_scale)^2
 * Parameters: one float array in the order W1, b1, W2, b2, ..., W7, b7,
 * each W in [Cout][3][3][3][Cin] with (Cin, Cout) = (16,16), (16,32),
 * (32,64), (64,128), (128,64), (64,64), (64,16); ngf_net_param_count gives
 * its length.  Training: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on a float
 * master copy with a bf16 copy for the tensor cores.
 * R, T: device float [B][s^3] (x fastest); u, u_target: device float
 * [B][3][Nn]; params and grads: host or device float arrays.  Calls enqueue
 * on the net's stream; those with a host loss synchronise it. */
typedef struct {
    int32_t s;          /* input images s^3, s a multiple of 8 in [8, 512] */
    int32_t max_batch;  /* pairs per call, >= 1 (workspace is sized for it) */
    float in_shift;     /* input normalisation: (I - in_shift) * in_scale  */
    float in_scale;
    float out_scale;    /* output scale (units of u), > 0                   */
} ngf_net_desc;
typedef struct ngf_net ngf_net;

int64_t ngf_net_param_count(const ngf_net_desc* desc);  /* -1 for a bad desc */
ngf_status ngf_net_create(ngf_net** net, const ngf_net_desc* desc, void* cuda_stream);
ngf_status ngf_net_destroy(ngf_net* net);
/* Copy all parameters in (resets the Adam moments and step) or out. */
ngf_status ngf_net_set_params(ngf_net* net, const float* params);
ngf_status ngf_net_get_params(ngf_net* net, float* params);
/* u = network(R, T) for B <= max_batch pairs. */
ngf_status ngf_net_forward(ngf_net* net, const float* R, const float* T, int32_t B, float* u);
/* Loss and its gradient with respect to every parameter (no update);
 * grads nullable, loss (host) nullable. */
ngf_status ngf_net_grad(ngf_net* net, const float* R, const float* T, const float* u_target, int32_t B,
                        float* grads, double* loss);
/* One training step: forward, backward, Adam update with learning rate lr;
 * loss (host, the loss before the update) nullable (then no sync). */
ngf_status ngf_net_train_step(ngf_net* net, const float* R, const float* T, const float* u_target, int32_t B,
                              double lr, double* loss);

/* Training loop: one Adam step per batch of `batch` consecutive entries of
 * order[0 .. count-1] (pair indices into R, T [npairs][s^3] and u_target
 * [npairs][3][Nn], device), each batch gathered into the net's staging
 * buffers by device copies; losses (host, nullable): the loss of each
 * batch before its update, ceil(count / batch) doubles.  Synchronises. */
ngf_status ngf_net_train(ngf_net* net, const float* R, const float* T, const float* u_target, int32_t npairs,
                         const int32_t* order, int32_t count, int32_t batch, double lr, double* losses);

/* Synchronises `cuda_stream` and returns the number of bounded waits of the
 * convolution kernels that gave up since the last call (0 in a healthy run;
 * a kernel that gives up leaves its output undefined but frees what it holds
 * and returns), or a negative ngf_status if the synchronisation failed. */
int32_t ngf_conv3d_check(void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NGF_CNN_H */
