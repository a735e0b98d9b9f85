// 3x3x3 convolution as an implicit GEMM on the tcgen05 tensor cores.
//
// GEMM view: rows m = output voxels (B*D*H*W), columns n = output channels,
// reduction k = (tap, input channel), 27*Cin long.  A CTA owns 128
// consecutive voxels and all Cout channels: one tcgen05.mma of shape
// M=128 x N=Cout x K=16 per 16 channels of a tap, FP32 accumulator in tensor
// memory (Cout columns x 128 lanes).  The reduction runs in stages of one tap
// x up to 64 channels through 3-6 shared-memory buffers: the 128 threads
// start asynchronous 16-byte copies (cp.async, zero fill outside the volume)
// of the stages ahead while the tensor core works on the current one, and
// one mbarrier per buffer, signalled by tcgen05.commit, tells them when a
// buffer may be refilled.
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
#include "ngf_plan.h"

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
    int tps;          // taps per stage: 1 (4 taps of 16 channels per stage
                      // measured slower: fewer CTAs fit on an SM)
    int nbuf;         // operand buffers in shared memory (3 .. CONV_MAXBUF)
    int ns;           // output channels per CTA (blockIdx.y selects the slice)
};

constexpr int CONV_MAXBUF = 6;

// Byte offset of 16-byte chunk q (channels 8q..8q+7 of the stage) of row r
// in a K-major, no-swizzle operand with `rows` rows.
__device__ __forceinline__ uint32_t operand_off(int r, int q, int rows) {
    return (uint32_t)((q >> 1) * (rows / 8) * 256 + (r >> 3) * 256 + (q & 1) * 128 + (r & 7) * 16);
}

// 16-byte asynchronous copy global -> shared; src_bytes = 0 writes zeros
// and reads nothing.
__device__ __forceinline__ void cp16_ca(uint32_t dst, const void* src, uint32_t src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp16_cg(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__global__ void __launch_bounds__(CONV_THREADS) k_conv3d_fwd(const ConvArgs a) {
    NGF_DYNAMIC_SMEM(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbuf = a.nbuf;
    const int kstage = a.tps * a.kst;  // reduction length of one stage
    const int ns = a.ns, n0 = blockIdx.y * a.ns;  // this CTA's output channels
    const uint32_t a_bytes = CONV_M * kstage * 2, b_bytes = ns * kstage * 2;
    const uint32_t sA = smem_addr(smem), sB = sA + nbuf * a_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + nbuf * (a_bytes + b_bytes));
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + CONV_MAXBUF);
    uint32_t ncols = 32;
    while ((int)ncols < ns) ncols <<= 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < nbuf; ++i) mbar_init(smem_addr(&bars[i]), 1);
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
    const int qn = a.kst / 8;  // 16-byte chunks per row per tap of a stage
    const int stages = ((27 + a.tps - 1) / a.tps) * a.cchunks;
    const uint32_t idesc = instr_desc(CONV_M, ns);
    bool failed = false;

    // start the copies of stage t into buffer t % nbuf
    auto load_stage = [&](int t) {
        const int buf = t % nbuf;
        const int tap0 = (t / a.cchunks) * a.tps, c0 = (t % a.cchunks) * a.kst;
        const int ntap = min(a.tps, 27 - tap0);
        // A: this thread's row, channels c0..c0+kst-1 of each shifted voxel
        // (8 lanes of a shared-memory phase write 8 rows of one core matrix)
        const uint32_t dA = sA + buf * a_bytes;
        for (int i = 0; i < ntap; ++i) {
            const int tap = tap0 + i;
            const int xx = vx + tap % 3 - 1, yy = vy + (tap / 3) % 3 - 1, zz = vz + tap / 9 - 1;
            const bool in = row_ok && xx >= 0 && xx < a.W && yy >= 0 && yy < a.H && zz >= 0 && zz < a.D;
            const uint4* src = a.x;
            if (in) src += ((((vb * a.D + zz) * a.H + yy) * a.W + xx) * a.cin + c0) / 8;
            for (int q = 0; q < qn; ++q)
                cp16_ca(dA + operand_off(tid, i * qn + q, CONV_M), in ? src + q : a.x, in ? 16u : 0u);
        }
        // B: this CTA's ns output channels, the same channels of the same taps
        const uint32_t dB = sB + buf * b_bytes;
        const int per_row = ntap * qn;
        for (int idx = tid; idx < ns * per_row; idx += CONV_THREADS) {
            const int n = idx / per_row, r = idx - n * per_row, i = r / qn, q = r - i * qn;
            cp16_cg(dB + operand_off(n, r, ns),
                    a.w + (((long long)(n0 + n) * 27 + tap0 + i) * a.cin + c0) / 8 + q);
        }
    };

    // copies run nbuf-2 stages ahead of the tensor core; a buffer is reused
    // once the MMAs of the stage two before the current one have completed
    const int ahead = nbuf - 2;
    for (int t = 0; t < ahead && t < stages; ++t) {
        load_stage(t);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int s = 0; s < stages; ++s) {
        const int t = s + ahead;
        if (t < stages) {
            if (t >= nbuf) {
                // buffer t % nbuf was read by the MMAs of stage t - nbuf = s - 2
                const bool ok = mbar_wait(smem_addr(&bars[t % nbuf]), (uint32_t)(((t - nbuf) / nbuf) & 1));
                if (__syncthreads_or(!ok)) { failed = true; break; }
            }
            load_stage(t);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        // all groups but the newest `ahead` ones are complete: stage s is in
        switch (ahead) {
            case 1: asm volatile("cp.async.wait_group 1;" ::: "memory"); break;
            case 2: asm volatile("cp.async.wait_group 2;" ::: "memory"); break;
            case 3: asm volatile("cp.async.wait_group 3;" ::: "memory"); break;
            default: asm volatile("cp.async.wait_group 4;" ::: "memory"); break;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int buf = s % nbuf;
            const uint32_t abase = sA + buf * a_bytes, bbase = sB + buf * b_bytes;
            const int slabs = min(a.tps, 27 - (s / a.cchunks) * a.tps) * a.kst / 16;
            for (int j = 0; j < slabs; ++j) {
                const uint64_t ad = smem_desc(abase + j * (CONV_M / 8) * 256, 128, 256);
                const uint64_t bd = smem_desc(bbase + j * (ns / 8) * 256, 128, 256);
                mma_bf16(tmem, ad, bd, idesc, (s > 0 || j > 0) ? 1u : 0u);
            }
            mma_commit(smem_addr(&bars[buf]));
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");

    // wait for the last commit of each buffer (all MMAs complete)
    bool ok = !failed;
    for (int s = stages - nbuf; s < stages && !failed; ++s) {
        if (s < 0) continue;
        ok &= mbar_wait(smem_addr(&bars[s % nbuf]), (uint32_t)((s / nbuf) & 1));
    }
    if (__syncthreads_or(!ok)) failed = true;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!failed) {
        // epilogue: warp w holds TMEM lanes 32w..32w+31 = rows of this CTA
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float* out = a.y + (row_ok ? v * a.cout + n0 : 0);
        for (int c = 0; c < ns; c += 16) {
            float r[16];
            tmem_load16(tmem + lane_base + (uint32_t)c, r);
            if (row_ok) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    float t = r[i] + (a.bias ? a.bias[n0 + c + i] : 0.0f);
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
        mbar_wait(smem_addr(&bars[(stages - 1) % nbuf]), (uint32_t)(((stages - 1) / nbuf) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ---- brick form (Cin <= 64): the input tile is staged once ---------------
//
// A CTA owns an 8 (x) x 16 (y) x P (z) block of output voxels: P MMA row
// tiles of 128 (row m = voxel (m & 7, m >> 3) of a plane), P accumulators of
// ncols tensor-memory columns each.  The (8+2) x (16+2) x (P+2) input brick
// with all Cin channels is copied to shared memory once, stored channel
// group major ([Cin/8][z][y][x], 16 bytes per voxel and group), so that the
// operand of tap (dz, dy, dx) is the brick itself at a start address moved
// by (dz, dy, dx) voxels: rows of a core matrix are 8 consecutive x (16
// bytes apart), 8-row groups are brick lines (stride 160 bytes), and the two
// channel groups of a K=16 slab are one channel-group plane apart.  No input
// voxel is gathered twice; only the weights stream, one tap per stage,
// shared by the P planes.

constexpr int BR_X = 10, BR_Y = 18;  // brick extent in x and y (tile + halo)

struct BrickArgs {
    const uint4* x;
    const uint4* w;
    const float* bias;
    float* y;
    int B, D, H, W, cin, cout, relu;
    int P;            // output planes per CTA
    int ncols;        // tensor-memory columns per accumulator
    int nbuf;         // weight buffers (3 .. CONV_MAXBUF)
    int tiles_x, tiles_y, tiles_z;
};

// Weights of tap s repacked into the exact shared-memory image of the B
// operand (K-major core matrices), so that one bulk copy moves a whole stage.
__global__ void k_conv3d_pack_w(const uint4* __restrict__ w, uint4* __restrict__ wp, int cout, int qn) {
    const int per_tap = cout * qn;
    const int total = 27 * per_tap;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
        const int s = idx / per_tap, r = idx - s * per_tap, n = r / qn, q = r - n * qn;
        wp[(size_t)s * per_tap + operand_off(n, q, cout) / 16] = w[((size_t)n * 27 + s) * qn + q];
    }
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Roles after the brick is staged: thread 32 (warp 1) streams the packed
// weights, one bulk copy per tap, into nbuf buffers (a "full" mbarrier per
// buffer counts the bytes); thread 0 issues the MMAs of each tap once its
// buffer is full and commits to the buffer's "empty" mbarrier, and after
// the last tap to the "done" mbarrier that the whole CTA waits on.
__global__ void __launch_bounds__(CONV_THREADS) k_conv3d_brick(const BrickArgs a) {
    NGF_DYNAMIC_SMEM(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbuf = a.nbuf, P = a.P, cg = a.cin / 8;
    const int nb = BR_X * BR_Y * (P + 2);           // brick voxels
    const uint32_t brick_bytes = (uint32_t)cg * nb * 16, b_bytes = (uint32_t)a.cout * a.cin * 2;
    const uint32_t sBr = smem_addr(smem), sB = sBr + brick_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + brick_bytes + nbuf * b_bytes);
    uint64_t* empty = full + CONV_MAXBUF;
    uint64_t* done = empty + CONV_MAXBUF;
    int* flags = reinterpret_cast<int*>(done + 1);  // [0] failed, [1] copies issued, [2] taps consumed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(flags + 3);
    const uint32_t tcols = (uint32_t)(P * a.ncols);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < nbuf; ++i) {
            mbar_init(smem_addr(&full[i]), 1);
            mbar_init(smem_addr(&empty[i]), 1);
        }
        mbar_init(smem_addr(done), 1);
        flags[0] = 0; flags[1] = 0; flags[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    int t = blockIdx.x;
    const int tx = t % a.tiles_x; t /= a.tiles_x;
    const int ty = t % a.tiles_y; t /= a.tiles_y;
    const int tz = t % a.tiles_z;
    const int b = t / a.tiles_z;
    const int x0 = tx * 8, y0 = ty * 16, z0 = tz * P;

    // the brick: one 16-byte copy per (voxel, channel group), channel group
    // fastest across lanes (contiguous global reads), zero outside
    for (int idx = tid; idx < cg * nb; idx += CONV_THREADS) {
        const int g = idx % cg, v = idx / cg;
        const int bx = v % BR_X, by = (v / BR_X) % BR_Y, bz = v / (BR_X * BR_Y);
        const int gx = x0 - 1 + bx, gy = y0 - 1 + by, gz = z0 - 1 + bz;
        const bool in = gx >= 0 && gx < a.W && gy >= 0 && gy < a.H && gz >= 0 && gz < a.D;
        const uint4* src = a.x;
        if (in) src += ((((long long)b * a.D + gz) * a.H + gy) * a.W + gx) * cg + g;
        cp16_ca(sBr + (uint32_t)(g * nb + v) * 16, src, in ? 16u : 0u);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (tid == 32) {
        // weight producer
        const unsigned char* wp = reinterpret_cast<const unsigned char*>(a.w);
        for (int s = 0; s < 27; ++s) {
            const int buf = s % nbuf;
            if (s >= nbuf && !mbar_wait(smem_addr(&empty[buf]), (uint32_t)(((s - nbuf) / nbuf) & 1))) {
                atomicExch(&flags[0], 1);
                break;
            }
            if (*(volatile int*)&flags[0]) break;
            mbar_expect_tx(smem_addr(&full[buf]), b_bytes);
            bulk_copy(sB + buf * b_bytes, wp + (size_t)s * b_bytes, b_bytes, smem_addr(&full[buf]));
            flags[1] = s + 1;
        }
    } else if (tid == 0) {
        // MMA issuer
        const uint32_t idesc = instr_desc(CONV_M, a.cout);
        const uint32_t lbo = (uint32_t)nb * 16;  // one channel group plane
        for (int s = 0; s < 27; ++s) {
            const int buf = s % nbuf;
            if (!mbar_wait(smem_addr(&full[buf]), (uint32_t)((s / nbuf) & 1))) {
                atomicExch(&flags[0], 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int dz = s / 9, dy = (s / 3) % 3, dx = s % 3;  // brick offsets 0..2
            const uint32_t bbase = sB + buf * b_bytes;
            for (int p = 0; p < P; ++p) {
                const uint32_t abase = sBr + (uint32_t)(((p + dz) * BR_Y + dy) * BR_X + dx) * 16;
                for (int j = 0; j < a.cin / 16; ++j) {
                    const uint64_t ad = smem_desc(abase + 2 * j * lbo, lbo, BR_X * 16);
                    const uint64_t bd = smem_desc(bbase + j * (a.cout / 8) * 256, 128, 256);
                    mma_bf16(tmem + (uint32_t)(p * a.ncols), ad, bd, idesc, (s > 0 || j > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_addr(&empty[buf]));
            flags[2] = s + 1;
        }
        mma_commit(smem_addr(done));  // all MMAs issued above are complete
    }
    __syncwarp();
    const bool ok = mbar_wait(smem_addr(done), 0u);
    __syncthreads();
    const bool failed = __syncthreads_or(!ok || flags[0] != 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (!failed) {
        const int m = warp * 32 + (tid & 31);
        const int vx = x0 + (m & 7), vy = y0 + (m >> 3);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int p = 0; p < P; ++p) {
            const int vz = z0 + p;
            const bool row_ok = vx < a.W && vy < a.H && vz < a.D;
            float* out = a.y + (row_ok ? ((((long long)b * a.D + vz) * a.H + vy) * a.W + vx) * a.cout : 0);
            for (int c = 0; c < a.cout; c += 16) {
                float r[16];
                tmem_load16(tmem + lane_base + (uint32_t)(p * a.ncols + c), r);
                if (row_ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float v = r[i] + (a.bias ? a.bias[c + i] : 0.0f);
                        r[i] = (a.relu && v < 0.0f) ? 0.0f : v;
                    }
#pragma unroll
                    for (int i = 0; i < 16; i += 4)
                        *reinterpret_cast<float4*>(out + c + i) = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
                }
            }
        }
    } else if (tid == 0) {
        atomicAdd(&g_conv_timeouts, 1u);
        // bounded waits for bulk copies still in flight (issued, not consumed)
        for (int s = flags[2]; s < flags[1]; ++s) mbar_wait(smem_addr(&full[s % nbuf]), (uint32_t)((s / nbuf) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
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
    int ncols = 32;
    while (ncols < Cout) ncols <<= 1;
    const size_t per_sm = 228 * 1024;
    if (Cin <= CONV_KMAX) {
        // brick form: P output planes per CTA, as many as leave room for two
        // CTAs per SM (256 tensor-memory columns, about 110 KB of shared
        // memory each): a second CTA stages its brick and drains its
        // accumulators while the other one's MMAs run (measured faster than
        // twice the planes in one CTA per SM)
        BrickArgs br;
        br.x = static_cast<const uint4*>(x);
        br.w = static_cast<const uint4*>(w);
        br.bias = bias;
        br.y = y;
        br.B = B; br.D = D; br.H = H; br.W = W;
        br.cin = Cin; br.cout = Cout; br.relu = relu ? 1 : 0;
        br.ncols = ncols;
        const size_t wst = (size_t)Cout * Cin * 2;
        br.P = 1;
        br.nbuf = 3;
        for (int p = 4; p >= 1; p >>= 1) {
            if (p * ncols > 256 || (p > 1 && p > D)) continue;
            const size_t brick = (size_t)(Cin / 8) * BR_X * BR_Y * (p + 2) * 16;
            int nbf = CONV_MAXBUF;
            while (nbf > 3 && brick + nbf * wst > 110 * 1024) --nbf;
            if (brick + nbf * wst <= 110 * 1024 || p == 1) { br.P = p; br.nbuf = nbf; break; }
        }
        br.tiles_x = (W + 7) / 8;
        br.tiles_y = (H + 15) / 16;
        br.tiles_z = (D + br.P - 1) / br.P;
        const size_t brick = (size_t)(Cin / 8) * BR_X * BR_Y * (br.P + 2) * 16;
        size_t smem = brick + br.nbuf * wst + (2 * CONV_MAXBUF + 1) * sizeof(uint64_t) + 32;
        // every resident CTA's tensor-memory allocation must fit at once
        const size_t ctas = 512 / (br.P * ncols);
        const size_t smem_min = per_sm / (ctas + 1) - 1024 + 16;
        if (smem < smem_min) smem = smem_min;
        const long long grid = (long long)br.tiles_x * br.tiles_y * br.tiles_z * B;
        if (grid >= (1LL << 31) || smem > 200 * 1024) return NGF_EBOUNDS;
        static bool battr = false;
        if (!battr) {
            if (cudaFuncSetAttribute(k_conv3d_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
                cudaSuccess)
                return NGF_ECUDA;
            battr = true;
        }
        // weights repacked per tap into the B operand's shared-memory image
        cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
        void* wp = nullptr;
        if (dev_alloc(&wp, 27 * wst, st) != cudaSuccess) return NGF_ENOMEM;
        const int chunks = 27 * Cout * (Cin / 8);
        const bool ok = launch(k_conv3d_pack_w, dim3((chunks + 255) / 256), dim3(256), 0, st,
                               static_cast<const uint4*>(w), static_cast<uint4*>(wp), (int)Cout,
                               (int)(Cin / 8)) == cudaSuccess &&
                        (br.w = static_cast<const uint4*>(wp),
                         launch(k_conv3d_brick, dim3((unsigned)grid), dim3(CONV_THREADS), smem, st, br) ==
                             cudaSuccess);
        dev_free(wp, st);
        return ok ? NGF_OK : NGF_ECUDA;
    }
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
    a.tps = 1;
    // output channels per CTA: split Cout while the grid is under two CTAs
    // per SM (small volumes)
    const long long gridm = (V + CONV_M - 1) / CONV_M;
    a.ns = Cout;
    while (a.ns % 32 == 0 && gridm * (Cout / a.ns) < 2 * 148) a.ns /= 2;
    ncols = 32;
    while (ncols < a.ns) ncols <<= 1;
    const size_t stage_bytes = ((size_t)CONV_M + a.ns) * a.tps * a.kst * 2;
    a.nbuf = CONV_MAXBUF;
    while (a.nbuf > 3 && a.nbuf * stage_bytes > 112 * 1024) --a.nbuf;
    size_t smem = a.nbuf * stage_bytes + CONV_MAXBUF * sizeof(uint64_t) + 16;
    // at most 512 / ncols CTAs per SM, so that every CTA's tensor-memory
    // allocation succeeds at once (228 KB of shared memory per SM, 1 KB of
    // it reserved per CTA)
    const size_t ctas = 512 / ncols;
    const size_t smem_min = per_sm / (ctas + 1) - 1024 + 16;
    if (smem < smem_min) smem = smem_min;
    static bool attr_set = false;
    if (!attr_set) {
        if (cudaFuncSetAttribute(k_conv3d_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
            return NGF_ECUDA;
        attr_set = true;
    }
    if (gridm >= (1LL << 31)) return NGF_EBOUNDS;
    if (launch(k_conv3d_fwd, dim3((unsigned)gridm, (unsigned)(Cout / a.ns)), dim3(CONV_THREADS), smem,
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
