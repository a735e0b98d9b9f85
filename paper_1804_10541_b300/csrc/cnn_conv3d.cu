// 3x3x3 convolution as an implicit GEMM on the tcgen05 tensor cores.
//
// GEMM view: rows m = output voxels (B*D*H*W), columns n = output channels,
// reduction k = (tap, input channel), 27*Cin long.  A CTA owns 128
// consecutive voxels and all Cout channels: one tcgen05.mma of shape
// M=128 x N=Cout x K=16 per 16 channels of a tap, FP32 accumulator in tensor
// memory (Cout columns x 128 lanes).  The reduction runs in stages of one tap
// x up to 64 channels, double-buffered in shared memory: the 128 threads
// gather the next stage (plain 16-byte loads; zero outside the volume) while
// the tensor core works on the current one, and an mbarrier signalled by
// tcgen05.commit tells them when a buffer may be overwritten.
//
// Shared-memory operand layout (K-major, no swizzle): 8x8 core matrices of
// 16-byte rows; within one K=16 slab the two K-halves of a row group are
// 128 bytes apart (leading byte offset) and consecutive 8-row groups 256
// bytes apart (stride byte offset).
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>

#include "ngf.h"
#include "ngf_cnn.h"
#include "ngf_launch.cuh"

namespace ngf {
namespace {

constexpr int CONV_M = 128;        // voxels per CTA (MMA M)
constexpr int CONV_THREADS = 128;  // 4 warps: one TMEM lane quarter each
constexpr int CONV_KMAX = 64;      // channels per stage
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // mbarrier polls before giving up

__device__ unsigned int g_conv_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start, leading and stride byte offsets
// (16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N/8 and M/16.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait for the completion of phase `parity`; false if it gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
            " selp.b32 %0, 1, 0, P;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_load16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct ConvArgs {
    const uint4* x;   // bf16 activations, 8 channels per uint4
    const uint4* w;   // bf16 weights, 8 channels per uint4
    const float* bias;
    float* y;
    int B, D, H, W, cin, cout, relu;
    long long V;      // B*D*H*W
    int kst;          // channels per stage
    int cchunks;      // stages per tap
};

// Byte offset of 16-byte chunk q (channels 8q..8q+7 of the stage) of row r
// in a K-major, no-swizzle operand with `rows` rows.
__device__ __forceinline__ uint32_t operand_off(int r, int q, int rows) {
    return (uint32_t)((q >> 1) * (rows / 8) * 256 + (r >> 3) * 256 + (q & 1) * 128 + (r & 7) * 16);
}

__global__ void __launch_bounds__(CONV_THREADS) k_conv3d_fwd(const ConvArgs a) {
    NGF_DYNAMIC_SMEM(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t a_bytes = CONV_M * a.kst * 2, b_bytes = a.cout * a.kst * 2;
    unsigned char* bufA[2] = {smem, smem + a_bytes};
    unsigned char* bufB[2] = {smem + 2 * a_bytes, smem + 2 * a_bytes + b_bytes};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 2 * a_bytes + 2 * b_bytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    uint32_t ncols = 32;
    while ((int)ncols < a.cout) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_addr(&bars[0]), 1);
        mbar_init(smem_addr(&bars[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    // this thread's output row (voxel) and its coordinates
    const long long v = (long long)blockIdx.x * CONV_M + tid;
    const bool row_ok = v < a.V;
    int vx = 0, vy = 0, vz = 0;
    long long vb = 0;
    if (row_ok) {
        long long t = v;
        vx = (int)(t % a.W); t /= a.W;
        vy = (int)(t % a.H); t /= a.H;
        vz = (int)(t % a.D); vb = t / a.D;
    }
    const int qn = a.kst / 8;  // 16-byte chunks per row per stage
    const int stages = 27 * a.cchunks;
    const uint32_t idesc = instr_desc(CONV_M, a.cout);
    bool failed = false;

    for (int s = 0; s < stages; ++s) {
        const int buf = s & 1;
        if (s >= 2) {
            // the MMAs of stage s-2 read this buffer: wait for their commit
            const bool ok = mbar_wait(smem_addr(&bars[buf]), (uint32_t)(((s - 2) >> 1) & 1));
            if (__syncthreads_or(!ok)) { failed = true; break; }
        }
        const int tap = s / a.cchunks, c0 = (s % a.cchunks) * a.kst;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        // A: this thread's row, channels c0..c0+kst-1 of the shifted voxel
        {
            const int xx = vx + dx, yy = vy + dy, zz = vz + dz;
            const bool in = row_ok && xx >= 0 && xx < a.W && yy >= 0 && yy < a.H && zz >= 0 && zz < a.D;
            const uint4* src = a.x;
            if (in) src += ((((vb * a.D + zz) * a.H + yy) * a.W + xx) * a.cin + c0) / 8;
            for (int q = 0; q < qn; ++q) {
                uint4 val = in ? src[q] : make_uint4(0u, 0u, 0u, 0u);
                *reinterpret_cast<uint4*>(bufA[buf] + operand_off(tid, q, CONV_M)) = val;
            }
        }
        // B: all Cout rows, same channels of the same tap
        for (int idx = tid; idx < a.cout * qn; idx += CONV_THREADS) {
            const int n = idx / qn, q = idx - n * qn;
            const uint4 val = a.w[(((long long)n * 27 + tap) * a.cin + c0) / 8 + q];
            *reinterpret_cast<uint4*>(bufB[buf] + operand_off(n, q, a.cout)) = val;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t abase = smem_addr(bufA[buf]), bbase = smem_addr(bufB[buf]);
            for (int j = 0; j < a.kst / 16; ++j) {
                const uint64_t ad = smem_desc(abase + j * (CONV_M / 8) * 256, 128, 256);
                const uint64_t bd = smem_desc(bbase + j * (a.cout / 8) * 256, 128, 256);
                mma_bf16(tmem, ad, bd, idesc, (s > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(smem_addr(&bars[buf]));
        }
    }

    // wait for the last commit of each buffer (all MMAs complete)
    bool ok = !failed;
    for (int s = stages - 2; s < stages && !failed; ++s) {
        if (s < 0) continue;
        ok &= mbar_wait(smem_addr(&bars[s & 1]), (uint32_t)((s >> 1) & 1));
    }
    if (__syncthreads_or(!ok)) failed = true;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!failed) {
        // epilogue: warp w holds TMEM lanes 32w..32w+31 = rows of this CTA
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float* out = a.y + (row_ok ? v * a.cout : 0);
        for (int c = 0; c < a.cout; c += 16) {
            float r[16];
            tmem_load16(tmem + lane_base + (uint32_t)c, r);
            if (row_ok) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float t = r[i] + (a.bias ? a.bias[c + i] : 0.0f);
                    r[i] = (a.relu && t < 0.0f) ? 0.0f : t;
                }
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(out + c + i) = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
            }
        }
    } else if (tid == 0) {
        atomicAdd(&g_conv_timeouts, 1u);
        // give MMAs still in flight a bounded chance to finish before the
        // tensor memory is released
        mbar_wait(smem_addr(&bars[(stages - 1) & 1]), (uint32_t)(((stages - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

}  // namespace
}  // namespace ngf

using namespace ngf;

extern "C" ngf_status ngf_conv3d_fwd(const void* x, const void* w, const float* bias, float* y, int32_t B,
                                     int32_t D, int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t relu,
                                     void* cuda_stream) {
    if (B < 0 || D < 0 || H < 0 || W < 0) return NGF_EINVAL;
    if (Cin < 16 || Cin % 16 != 0 || (Cin > CONV_KMAX && Cin % CONV_KMAX != 0)) return NGF_EINVAL;
    if (Cout < 16 || Cout > 256 || Cout % 16 != 0) return NGF_EINVAL;
    const long long V = (long long)B * D * H * W;
    if (V >= (1LL << 31)) return NGF_EBOUNDS;
    if (V == 0) return NGF_OK;
    if (!x || !w || !y) return NGF_EINVAL;
    if (((uintptr_t)x | (uintptr_t)w | (uintptr_t)y) & 15u) return NGF_EINVAL;
    ConvArgs a;
    a.x = static_cast<const uint4*>(x);
    a.w = static_cast<const uint4*>(w);
    a.bias = bias;
    a.y = y;
    a.B = B; a.D = D; a.H = H; a.W = W;
    a.cin = Cin; a.cout = Cout; a.relu = relu ? 1 : 0;
    a.V = V;
    a.kst = Cin <= CONV_KMAX ? Cin : CONV_KMAX;
    a.cchunks = Cin / a.kst;
    size_t smem = 2 * (size_t)CONV_M * a.kst * 2 + 2 * (size_t)Cout * a.kst * 2 + 2 * sizeof(uint64_t) + 16;
    // at most 512 / ncols CTAs per SM, so that every CTA's tensor-memory
    // allocation succeeds at once (228 KB of shared memory per SM, 1 KB of
    // it reserved per CTA)
    int ncols = 32;
    while (ncols < Cout) ncols <<= 1;
    const size_t per_sm = 228 * 1024, ctas = 512 / ncols;
    const size_t smem_min = per_sm / (ctas + 1) - 1024 + 16;
    if (smem < smem_min) smem = smem_min;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_conv3d_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024) !=
            cudaSuccess)
            return NGF_ECUDA;
        attr_set = true;
    }
    const long long grid = (V + CONV_M - 1) / CONV_M;
    if (launch(k_conv3d_fwd, dim3((unsigned)grid), dim3(CONV_THREADS), smem,
               static_cast<cudaStream_t>(cuda_stream), a) != cudaSuccess)
        return NGF_ECUDA;
    return NGF_OK;
}

extern "C" int32_t ngf_conv3d_check(void* cuda_stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) return NGF_ECUDA;
    unsigned int n = 0;
    if (cudaMemcpyFromSymbol(&n, g_conv_timeouts, sizeof(n)) != cudaSuccess) return NGF_ECUDA;
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_conv_timeouts, &zero, sizeof(zero)) != cudaSuccess) return NGF_ECUDA;
    return (int32_t)n;
}
