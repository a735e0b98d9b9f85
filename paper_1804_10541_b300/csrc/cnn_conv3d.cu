// 3x3x3 convolution as an implicit GEMM on the tcgen05 tensor cores.
//
// GEMM view: rows m = output voxels, columns n = output channels, reduction
// k = (tap, input channel), 27*Cin long.  One thread issues tcgen05.mma of
// shape M=128 x N x K=16 from shared-memory operands into FP32 accumulators
// in tensor memory; a second thread streams the weights by bulk copies;
// mbarriers (one "full" and one "empty" per weight buffer, signalled by the
// copy engine and by tcgen05.commit) order the two, and every wait on them
// is bounded.
//
// Shared-memory operand layout (K-major, no swizzle): 8x8 core matrices of
// 16-byte rows; the leading byte offset steps between the two 8-channel
// halves of a K=16 slab, the stride byte offset between 8-row groups.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <mutex>

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

// 16 columns of zeros into this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
        "r"(z)
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

// ---- brick form: the input tile is staged once per channel chunk ---------
//
// A CTA owns an 8 (x) x 16 (y) x P (z) block of output voxels and a slice
// of ns output channels (blockIdx.y): P MMA row tiles of 128 (row m = voxel
// (m & 7, m >> 3) of a plane), P accumulators of ncols tensor-memory columns
// each.  The input channels run in chunks of kc <= 64; for each chunk the
// (8+2) x (16+2) x (P+2) input brick is copied to shared memory once,
// stored channel group major ([kc/8][z][y][x], 16 bytes per voxel and
// group), so that the operand of tap (dz, dy, dx) is the brick itself at a
// start address moved by (dz, dy, dx) voxels: rows of a core matrix are 8
// consecutive x (16 bytes apart), 8-row groups are brick lines (stride 160
// bytes), and the two channel groups of a K=16 slab are one channel-group
// plane apart.  No input voxel is gathered twice per chunk; only the
// weights stream, one (chunk, tap) per stage, shared by the P planes.

constexpr int BR_X = 10, BR_Y = 18;  // brick extent in x and y (tile + halo)

struct BrickArgs {
    const uint4* x;
    const uint4* w;   // packed: [slice][chunk][tap] images of ns x kc
    const float* bias;
    void* y;          // float, or bf16 when out_bf16
    int B, D, H, W, cin, cout, relu, out_bf16;
    int P;            // output planes per CTA
    int ns;           // output channels per CTA
    int ncols;        // tensor-memory columns per accumulator
    int kc;           // input channels per chunk
    int nch;          // chunks
    int tps;          // taps per weight stage: 1, 3, 9 or 27
    int nbuf;         // weight buffers (1 .. CONV_MAXBUF)
    int tiles_x, tiles_y, tiles_z;
    int zs;           // z-stacked taps: one MMA per (dy, dx, input plane) with N = 3 ns
    int tcols;        // tensor-memory columns allocated
};

// Weights of (slice, chunk, tap) repacked into the exact shared-memory image
// of the B operand (K-major core matrices), so that one bulk copy moves a
// whole stage.  z-stacked (zs): one image per (slice, chunk, dy, dx) of
// 3 ns rows, row b ns + o holding tap (2 - b, dy, dx) of output channel o.
__device__ __forceinline__ void pack_index(long long idx, int ns, int qk, int nch, int zs, long long& dst, int& slice,
                                           int& chunk, int& tap, int& n, int& q) {
    const int rows = zs ? 3 * ns : ns, per_stage = rows * qk, nimg = zs ? 9 : 27;
    const long long st = idx / per_stage;  // (slice * nch + chunk) * nimg + image
    const int r = (int)(idx - st * per_stage), nr = r / qk;
    q = r - nr * qk;
    const int img = (int)(st % nimg);
    chunk = (int)((st / nimg) % nch);
    slice = (int)(st / ((long long)nimg * nch));
    n = zs ? nr % ns : nr;
    tap = zs ? (2 - nr / ns) * 9 + img : img;
    dst = st * per_stage + operand_off(nr, q, rows) / 16;
}

__global__ void k_conv3d_pack_w(const uint4* __restrict__ w, uint4* __restrict__ wp, int cout, int cin, int ns,
                                int kc, int zs) {
    const int qk = kc / 8, nch = cin / kc;
    const long long total = (long long)(cout / ns) * nch * 27 * ns * qk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long dst;
        int slice, chunk, tap, n, q;
        pack_index(idx, ns, qk, nch, zs, dst, slice, chunk, tap, n, q);
        wp[dst] = w[((long long)(slice * ns + n) * 27 + tap) * (cin / 8) + chunk * qk + q];
    }
}

// Data-gradient weights: the data gradient of y = conv(x, w) is the
// convolution of dy with the taps mirrored and the channel roles swapped,
// w'[c][tap][o] = w[o][26 - tap][c]; this packs w' (read element by element
// from the forward layout w[cout][27][cin]) into the same shared-memory image
// as k_conv3d_pack_w, for a convolution with cin' = cout and cout' = cin.
__global__ void k_conv3d_pack_wT(const __nv_bfloat16* __restrict__ w, uint4* __restrict__ wp, int cout_f,
                                 int cin_f, int ns, int kc, int zs) {
    const int cinp = cout_f, coutp = cin_f;  // channels of the mirrored convolution
    const int qk = kc / 8, nch = cinp / kc;
    const long long total = (long long)(coutp / ns) * nch * 27 * ns * qk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long dst;
        int slice, chunk, tap, n, q;
        pack_index(idx, ns, qk, nch, zs, dst, slice, chunk, tap, n, q);
        const int oc = slice * ns + n;  // output channel of the mirrored convolution = forward input channel
        uint32_t pk[4];
        for (int e = 0; e < 8; e += 2) {
            const int ic0 = chunk * kc + 8 * q + e;  // input channel = forward output channel
            const __nv_bfloat16 lo = w[((long long)ic0 * 27 + (26 - tap)) * cin_f + oc];
            const __nv_bfloat16 hi = w[((long long)(ic0 + 1) * 27 + (26 - tap)) * cin_f + oc];
            pk[e / 2] = (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
        }
        wp[dst] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
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

// Tiled tensor copy of one 5-D box (TMA) from global to shared memory,
// completing on mbarrier `bar` with its byte count; coordinates in elements,
// innermost first (channel, x, y, z, batch); boxes reaching outside the
// tensor are filled with zeros.
__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            int c4, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5, %6}], [%7];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
        : "memory");
}

// Shared-memory bytes of one channel-group plane of the brick (16 bytes per
// voxel), rounded up to 128 so that every plane starts a tensor copy on a
// 128-byte boundary.
__host__ __device__ constexpr uint32_t brick_plane_bytes(int P) {
    return ((uint32_t)BR_X * BR_Y * (P + 2) * 16 + 127u) & ~127u;
}

// Per chunk: thread 0 copies the chunk's input brick by one tensor copy per
// channel group (zeros outside the volume) and the CTA waits for it; thread
// 32 (warp 1) streams
// the chunk's packed weights, one bulk copy per tap, into nbuf buffers (a
// "full" mbarrier per buffer counts the bytes); thread 0 issues the MMAs of
// each tap once its buffer is full and commits to the buffer's "empty"
// mbarrier, and after the chunk's last tap to the "chunk" mbarrier that the
// whole CTA waits on before restaging the brick (or draining the result).
__global__ void __launch_bounds__(CONV_THREADS) k_conv3d_brick(const BrickArgs a,
                                                               const __grid_constant__ CUtensorMap xmap) {
    NGF_DYNAMIC_SMEM(smem_raw);
    // the brick starts on a 128-byte boundary (tensor-copy destination)
    unsigned char* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nbuf = a.nbuf, P = a.P, cg = a.kc / 8, ns = a.ns, n0 = blockIdx.y * a.ns;
    const int nb = BR_X * BR_Y * (P + 2);           // brick voxels
    const uint32_t gplane = brick_plane_bytes(P);   // one channel group of the brick
    // one B image: ns rows (a tap) or, z-stacked, 3 ns rows (the three dz of one (dy, dx))
    const int nimg = a.zs ? 9 : 27;  // B images per chunk
    const uint32_t brick_bytes = (uint32_t)cg * gplane, b_bytes = (uint32_t)(a.zs ? 3 : 1) * ns * a.kc * 2;
    const uint32_t st_bytes = a.tps * b_bytes;     // one weight stage
    const int spc = nimg / a.tps;                  // stages per chunk
    const uint32_t sBr = smem_addr(smem), sB = sBr + brick_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + brick_bytes + nbuf * st_bytes);
    uint64_t* empty = full + CONV_MAXBUF;
    uint64_t* chunk_bar = empty + CONV_MAXBUF;
    uint64_t* brick_bar = chunk_bar + 1;                 // the brick's tensor copies
    int* flags = reinterpret_cast<int*>(brick_bar + 1);  // [0] failed, [1] copies issued, [2] stages consumed
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(flags + 3);
    const uint32_t tcols = (uint32_t)a.tcols;

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
        mbar_init(smem_addr(chunk_bar), 1);
        mbar_init(smem_addr(brick_bar), 1);
        flags[0] = 0; flags[1] = 0; flags[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    int t = blockIdx.x;
    const int tx = t % a.tiles_x; t /= a.tiles_x;
    const int ty = t % a.tiles_y; t /= a.tiles_y;
    const int tz = t % a.tiles_z;
    const int b = t / a.tiles_z;
    const int x0 = tx * 8, y0 = ty * 16, z0 = tz * P;
    const unsigned char* wp = reinterpret_cast<const unsigned char*>(a.w) +
                              (size_t)blockIdx.y * a.nch * nimg * b_bytes;  // this slice's stages
    uint32_t tmem = 0;
    bool failed = false;
    int brick_pending = -1;  // chunk whose brick copy is issued and not seen complete
    __syncthreads();  // barriers and flags initialised before the producer's first copy
    if (a.zs) {  // z-stacked accumulators start at zero: every MMA accumulates
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t t0 = *tmem_slot + ((uint32_t)(warp * 32) << 16);
        for (uint32_t col = 0; col < tcols; col += 16) tmem_zero16(t0 + col);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }

    for (int c = 0; c < a.nch; ++c) {
        if (c > 0) {
            // all MMAs of the previous chunk have read the brick
            const bool ok = mbar_wait(smem_addr(chunk_bar), (uint32_t)((c - 1) & 1));
            if (__syncthreads_or(!ok || flags[0] != 0)) { failed = true; break; }
        }
        // weight producer, first part: when all of the chunk's stages fit the
        // buffers, they go out before the brick is staged (they depend on
        // nothing and their buffers are free: the previous chunk's MMAs have
        // all completed), so their copies overlap the staging (5-10% faster
        // on the small layers; with more stages than buffers, issuing the
        // first ones early measured 10% slower); the rest follow the barrier,
        // paced by the MMA thread's releases
        const int pre_end = spc * c + (spc <= nbuf ? spc : 0);
        auto produce = [&](int s0, int s1) {
            for (int s = s0; s < s1; ++s) {
                const int buf = s % nbuf;
                if (s >= nbuf && !mbar_wait(smem_addr(&empty[buf]), (uint32_t)(((s - nbuf) / nbuf) & 1))) {
                    atomicExch(&flags[0], 1);
                    break;
                }
                if (*(volatile int*)&flags[0]) break;
                mbar_expect_tx(smem_addr(&full[buf]), st_bytes);
                bulk_copy(sB + buf * st_bytes, wp + (size_t)s * st_bytes, st_bytes, smem_addr(&full[buf]));
                flags[1] = s + 1;
            }
        };
        if (tid == 32) produce(spc * c, pre_end);
        // the brick of chunk c: one tensor copy per channel group, the box
        // (8 channels, 10 x, 18 y, P+2 z) from (x0-1, y0-1, z0-1) of batch b,
        // zeros outside the volume; every thread waits for its bytes
        if (tid == 0) {
            mbar_expect_tx(smem_addr(brick_bar), (uint32_t)cg * nb * 16);
            for (int g = 0; g < cg; ++g)
                tma_load_5d(sBr + g * gplane, &xmap, c * a.kc + 8 * g, x0 - 1, y0 - 1, z0 - 1, b,
                            smem_addr(brick_bar));
        }
        brick_pending = c;
        const bool brick_ok = mbar_wait(smem_addr(brick_bar), (uint32_t)(c & 1));
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(!brick_ok)) {
            if (tid == 0) atomicExch(&flags[0], 1);
            failed = true;
            break;
        }
        brick_pending = -1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = *tmem_slot;

        if (tid == 32) {
            produce(pre_end, spc * c + spc);  // weight producer, second part
        } else if (tid == 0) {
            // MMA issuer
            const uint32_t idesc = instr_desc(CONV_M, a.zs ? 3 * ns : ns);
            const uint32_t lbo = gplane;  // one channel group plane
            // Descriptors of the brick's and the weight buffers' starts: an
            // operand at byte offset o (a multiple of 16) is the start's
            // descriptor plus o / 16, since the start-address field holds
            // address / 16 in 14 bits and shared addresses stay below 256 KB
            // (no carry out of the field).
            const uint64_t ad0 = smem_desc(sBr, lbo, BR_X * 16), bd0 = smem_desc(sB, 128, 256);
            const uint32_t ja = 2 * lbo / 16, jb = (uint32_t)((a.zs ? 3 : 1) * ns / 8) * 256 / 16,
                           nkj = (uint32_t)(a.kc / 16);
            for (int s = spc * c; s < spc * c + spc; ++s) {
                const int buf = s % nbuf;
                if (!mbar_wait(smem_addr(&full[buf]), (uint32_t)((s / nbuf) & 1))) {
                    atomicExch(&flags[0], 1);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int i = 0; i < a.tps; ++i) {
                    const int img = (s - spc * c) * a.tps + i;
                    const uint64_t bd = bd0 + (buf * st_bytes + i * b_bytes) / 16;
                    if (a.zs) {
                        // (dy, dx) = img: input plane pi meets dz = 2, 1, 0 (image rows
                        // 0, ns, 2 ns) for output planes pi - 2, pi - 1, pi, whose
                        // accumulators sit at columns (q + 2) ns: one MMA at pi ns
                        const int dy = img / 3, dx = img % 3;
                        uint64_t ad = ad0 + (uint32_t)(dy * BR_X + dx);  // 16 bytes per brick voxel
                        uint32_t d = tmem;
                        for (int pi = 0; pi < P + 2; ++pi, ad += BR_X * BR_Y, d += (uint32_t)ns)
                            for (uint32_t j = 0; j < nkj; ++j) mma_bf16(d, ad + j * ja, bd + j * jb, idesc, 1u);
                    } else {
                        const int dz = img / 9, dy = (img / 3) % 3, dx = img % 3;  // brick offsets 0..2
                        uint64_t ad = ad0 + (uint32_t)((dz * BR_Y + dy) * BR_X + dx);
                        uint32_t d = tmem;
                        for (int p = 0; p < P; ++p, ad += BR_X * BR_Y, d += (uint32_t)a.ncols)
                            for (uint32_t j = 0; j < nkj; ++j)
                                mma_bf16(d, ad + j * ja, bd + j * jb, idesc, (s > 0 || i > 0 || j > 0) ? 1u : 0u);
                    }
                }
                mma_commit(smem_addr(&empty[buf]));
                flags[2] = s + 1;
            }
            mma_commit(smem_addr(chunk_bar));  // all MMAs issued so far are complete
        }
        __syncwarp();
    }
    if (!failed) {
        const bool ok = mbar_wait(smem_addr(chunk_bar), (uint32_t)((a.nch - 1) & 1));
        failed = __syncthreads_or(!ok || flags[0] != 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tmem_slot;

    if (!failed) {
        const int m = warp * 32 + (tid & 31);
        const int vx = x0 + (m & 7), vy = y0 + (m >> 3);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        for (int p = 0; p < P; ++p) {
            const int vz = z0 + p;
            const bool row_ok = vx < a.W && vy < a.H && vz < a.D;
            const long long obase = row_ok ? ((((long long)b * a.D + vz) * a.H + vy) * a.W + vx) * a.cout + n0 : 0;
            for (int cc = 0; cc < ns; cc += 16) {
                float r[16];
                tmem_load16(tmem + lane_base + (uint32_t)((a.zs ? (p + 2) * ns : p * a.ncols) + cc), r);
                if (row_ok) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float v = r[i] + (a.bias ? a.bias[n0 + cc + i] : 0.0f);
                        r[i] = (a.relu && v < 0.0f) ? 0.0f : v;
                    }
                    if (a.out_bf16) {
                        uint32_t pk[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const __nv_bfloat162 h2 = __floats2bfloat162_rn(r[2 * i], r[2 * i + 1]);
                            pk[i] = *reinterpret_cast<const uint32_t*>(&h2);
                        }
                        uint4* out = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.y) + obase + cc);
                        out[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        out[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                    } else {
                        float* out = static_cast<float*>(a.y) + obase + cc;
#pragma unroll
                        for (int i = 0; i < 16; i += 4)
                            *reinterpret_cast<float4*>(out + i) = make_float4(r[i], r[i + 1], r[i + 2], r[i + 3]);
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicAdd(&g_conv_timeouts, 1u);
        // bounded waits for bulk copies still in flight (issued, not consumed)
        for (int s = flags[2]; s < flags[1]; ++s) mbar_wait(smem_addr(&full[s % nbuf]), (uint32_t)((s / nbuf) & 1));
        if (brick_pending >= 0) mbar_wait(smem_addr(brick_bar), (uint32_t)(brick_pending & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tcols) : "memory");
    }
}

// cuTensorMapEncodeTiled of the installed driver, looked up once through the
// runtime (the library does not link the driver library itself).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

// Tensor map of the brick kernel's input x[B][D][H][W][C] (bf16, channels
// fastest): 5-D (C, W, H, D, B), boxes of 8 channels x 10 x 18 x (P+2) x 1,
// zeros outside.  The strides are multiples of 16 bytes because C is a
// multiple of 16, and x is 16-byte aligned (both checked by the caller).
bool brick_map(CUtensorMap* map, const void* x, int B, int D, int H, int W, int C, int P) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dim[5] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D, (cuuint64_t)B};
    const cuuint64_t stride[4] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2,
                                  (cuuint64_t)D * H * W * C * 2};
    const cuuint32_t box[5] = {8, BR_X, BR_Y, (cuuint32_t)(P + 2), 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dim, stride, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The brick kernel's dynamic shared-memory limit is raised once per device
// (the attribute is per device), under a lock.
std::mutex g_brick_mu;
bool g_brick_attr[256] = {};

bool brick_attr_set() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return false;
    std::lock_guard<std::mutex> lock(g_brick_mu);
    if (!g_brick_attr[dev]) {
        if (cudaFuncSetAttribute(k_conv3d_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
            return false;
        g_brick_attr[dev] = true;
    }
    return true;
}

}  // namespace
}  // namespace ngf

using namespace ngf;

namespace ngf {
namespace {

// ---- weight gradient ------------------------------------------------------
//
// dw[o][tap][c] = sum_v dy[v][o] x[v + tap][c] is a GEMM with rows o (M),
// columns c (N) and the voxels as the reduction (K), one accumulator per
// tap.  A CTA owns one column group (an input-channel chunk of kc channels
// and a group of tg taps: tg * kc <= 256 tensor-memory columns) and a range
// of output tiles of 16 (x) x TY x TZ voxels, and accumulates over all its
// tiles in tensor memory.  Per tile, the dy tile and the x brick (tile plus
// a one-voxel halo, kc channels) are copied to shared memory once, both
// channel-group major with 16 bytes (8 channels) per voxel, which makes
// both operands MN-major: a core matrix is 8 consecutive voxels (K) x 8
// channels (M or N), 128 contiguous bytes.  The K = 16 slab of one MMA is
// one x line of the tile; the B operand of tap (dz, dy, dx) is the brick
// line moved by (dz, dy, dx) voxels.  M is 128 (output channels beyond cout
// read neighbouring shared memory and their accumulator lanes are never
// read).  The CTA's partial sums go to global memory and a second kernel
// adds the CTAs of each column group in a fixed order (deterministic).

constexpr int WG_TX = 16;

struct WgradArgs {
    const uint4* x;    // [V][cin / 8]
    const uint4* dy;   // [V][cout / 8]
    float* part;       // [split][ngroups][cout][gcols]
    int B, D, H, W, cin, cout;
    int kc;            // input channels per chunk (N of the MMA)
    int tg, ntg;       // taps per group, tap groups
    int ngroups;       // chunks x tap groups
    int gcols;         // tg * kc
    int tcols;         // tensor-memory columns allocated
    int TY, TZ;        // tile extent in y and z (x: WG_TX)
    int tiles_x, tiles_y, tiles_z, ntiles;
    int split;         // CTAs per column group
    uint32_t a_bytes;  // shared-memory bytes of the dy tile region (with slack)
};

// Instruction descriptor of kind::f16 with both operands MN-major
// ("transposed" A and B bits set), FP32 accumulator, BF16 inputs.
__host__ __device__ constexpr uint32_t instr_desc_mn(int m, int n) {
    return instr_desc(m, n) | (1u << 15) | (1u << 16);
}

__global__ void __launch_bounds__(CONV_THREADS) k_conv3d_wgrad(const WgradArgs a) {
    NGF_DYNAMIC_SMEM(smem);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int cgo = a.cout / 8, cgi = a.kc / 8;
    const int bx = WG_TX + 2, by = a.TY + 2, bz = a.TZ + 2, nbv = bx * by * bz;
    const int ntv = WG_TX * a.TY * a.TZ, lines = a.TY * a.TZ;
    const uint32_t sA = smem_addr(smem), sB = sA + a.a_bytes;
    const uint32_t b_bytes = (uint32_t)(cgi + 1) * nbv * 16;  // one channel-group plane of slack
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + a.a_bytes + b_bytes);
    int* flags = reinterpret_cast<int*>(bar + 1);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(flags + 2);

    const int grp = blockIdx.y, chunk = grp / a.ntg, tgi = grp % a.ntg;
    const int tap0 = tgi * a.tg, ntap = min(a.tg, 27 - tap0);
    const int t0 = (int)((long long)blockIdx.x * a.ntiles / a.split);
    const int t1 = (int)((long long)(blockIdx.x + 1) * a.ntiles / a.split);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tmem_slot)),
                     "r"((uint32_t)a.tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(smem_addr(bar), 1);
        flags[0] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t tmem = 0;
    bool failed = false;
    int issued = 0;  // tiles whose MMAs were committed
    for (int t = t0; t < t1; ++t) {
        if (t > t0) {
            // the previous tile's MMAs have read shared memory
            const bool ok = mbar_wait(smem_addr(bar), (uint32_t)((issued - 1) & 1));
            if (__syncthreads_or(!ok || flags[0] != 0)) { failed = true; break; }
        }
        int r = t;
        const int tx = r % a.tiles_x; r /= a.tiles_x;
        const int ty = r % a.tiles_y; r /= a.tiles_y;
        const int tz = r % a.tiles_z;
        const int b = r / a.tiles_z;
        const int x0 = tx * WG_TX, y0 = ty * a.TY, z0 = tz * a.TZ;
        // dy tile: voxel v = (z * TY + y) * 16 + x at ((v / 8) * cgo + g) * 128 + (v % 8) * 16
        for (int idx = tid; idx < ntv * cgo; idx += CONV_THREADS) {
            const int g = idx % cgo, v = idx / cgo;
            const int vx = v % WG_TX, vy = (v / WG_TX) % a.TY, vz = v / (WG_TX * a.TY);
            const int gx = x0 + vx, gy = y0 + vy, gz = z0 + vz;
            const bool in = gx < a.W && gy < a.H && gz < a.D;
            const uint4* src = a.dy;
            if (in) src += ((((long long)b * a.D + gz) * a.H + gy) * a.W + gx) * cgo + g;
            cp16_ca(sA + (uint32_t)(((v >> 3) * cgo + g) * 128 + (v & 7) * 16), src, in ? 16u : 0u);
        }
        // x brick of this chunk, channel-group planes of nbv voxels, zero outside
        for (int idx = tid; idx < nbv * cgi; idx += CONV_THREADS) {
            const int g = idx % cgi, v = idx / cgi;
            const int ux = v % bx, uy = (v / bx) % by, uz = v / (bx * by);
            const int gx = x0 - 1 + ux, gy = y0 - 1 + uy, gz = z0 - 1 + uz;
            const bool in = gx >= 0 && gx < a.W && gy >= 0 && gy < a.H && gz >= 0 && gz < a.D;
            const uint4* src = a.x;
            if (in) src += ((((long long)b * a.D + gz) * a.H + gy) * a.W + gx) * (a.cin / 8) + chunk * cgi + g;
            cp16_ca(sB + (uint32_t)(g * nbv + v) * 16, src, in ? 16u : 0u);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = *tmem_slot;
        if (tid == 0) {
            const uint32_t idesc = instr_desc_mn(128, a.kc);
            // no swizzle, MN-major as K-major: the stride byte offset steps
            // between core matrices along M/N, the leading byte offset along K
            const uint32_t a_mn = 128, a_k = (uint32_t)cgo * 128;
            const uint32_t b_mn = (uint32_t)nbv * 16, b_k = 128;
            for (int j = 0; j < ntap; ++j) {
                const int tap = tap0 + j;
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                for (int l = 0; l < lines; ++l) {
                    const int yy = l % a.TY, zz = l / a.TY;
                    const uint64_t ad = smem_desc(sA + (uint32_t)(2 * l * cgo) * 128, a_k, a_mn);
                    const uint64_t bd =
                        smem_desc(sB + (uint32_t)(((zz + dz) * by + (yy + dy)) * bx + dx) * 16, b_k, b_mn);
                    mma_bf16(tmem + (uint32_t)(j * a.kc), ad, bd, idesc, (t > t0 || l > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_addr(bar));
        }
        __syncwarp();
        ++issued;
    }
    if (!failed && issued > 0) {
        const bool ok = mbar_wait(smem_addr(bar), (uint32_t)((issued - 1) & 1));
        failed = __syncthreads_or(!ok || flags[0] != 0);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tmem_slot;
    if (!failed) {
        const int co = warp * 32 + (tid & 31);
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        float* out = a.part + (((long long)blockIdx.x * a.ngroups + grp) * a.cout + (co < a.cout ? co : 0)) * a.gcols;
        for (int c = 0; c < ntap * a.kc; c += 16) {
            float v[16];
            if (issued > 0) {
                tmem_load16(tmem + lane_base + (uint32_t)c, v);
            } else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.0f;
            }
            if (co < a.cout) {
#pragma unroll
                for (int i = 0; i < 16; i += 4)
                    *reinterpret_cast<float4*>(out + c + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
            }
        }
    } else if (tid == 0) {
        atomicAdd(&g_conv_timeouts, 1u);
        mbar_wait(smem_addr(bar), (uint32_t)((issued - 1) & 1));  // MMAs still in flight (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)a.tcols)
                     : "memory");
    }
}

// dw[o][tap][c] = sum over the split CTAs of their partial sums, in order.
__global__ void k_conv3d_wgrad_reduce(const float* __restrict__ part, float* __restrict__ dw, int cout, int cin,
                                      int kc, int tg, int ntg, int ngroups, int gcols, int split) {
    const long long total = (long long)cout * 27 * cin;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % cin), tap = (int)((i / cin) % 27), o = (int)(i / (27LL * cin));
        const int grp = (c / kc) * ntg + tap / tg, col = (tap % tg) * kc + c % kc;
        float acc = 0.0f;
        for (int s = 0; s < split; ++s) acc += part[(((long long)s * ngroups + grp) * cout + o) * gcols + col];
        dw[i] = acc;
    }
}

// db[o] = sum_v dy[v][o]: per block a float partial over a contiguous voxel
// range (thread o sums channel o), then the blocks in order.
__global__ void k_bias_grad_part(const __nv_bfloat16* __restrict__ dy, float* __restrict__ part, long long V,
                                 int cout, int per_block) {
    const long long v0 = (long long)blockIdx.x * per_block;
    const long long v1 = v0 + per_block < V ? v0 + per_block : V;
    for (int o = threadIdx.x; o < cout; o += blockDim.x) {
        float acc = 0.0f;
        for (long long v = v0; v < v1; ++v) acc += __bfloat162float(dy[v * cout + o]);
        part[(long long)blockIdx.x * cout + o] = acc;
    }
}

__global__ void k_bias_grad_sum(const float* __restrict__ part, float* __restrict__ db, int nblocks, int cout) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < cout; o += gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int k = 0; k < nblocks; ++k) acc += part[(long long)k * cout + o];
        db[o] = acc;
    }
}

std::mutex g_wg_mu;
bool g_wg_attr[256] = {};

bool wgrad_attr_set() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return false;
    std::lock_guard<std::mutex> lock(g_wg_mu);
    if (!g_wg_attr[dev]) {
        if (cudaFuncSetAttribute(k_conv3d_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess)
            return false;
        g_wg_attr[dev] = true;
    }
    return true;
}

// Brick-form convolution of x [V][cin] with packed weights: w is either the
// layer's own weights [cout][27][cin] or, when mirrored, the weights of a
// forward layer with cin_f = cout and cout_f = cin (the data gradient).
ngf_status conv_run(const void* x, const void* w, bool mirrored, const float* bias, void* y, bool out_bf16,
                    int32_t B, int32_t D, int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t relu,
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
    int dev = 0, sm_count = 0, smem_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return NGF_ECUDA;
    const size_t per_sm = (size_t)smem_sm;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    {
        // brick form: P output planes per CTA, as many as leave room for two
        // CTAs per SM (256 tensor-memory columns, about 110 KB of shared
        // memory each): a second CTA stages its brick and drains its
        // accumulators while the other one's MMAs run (measured faster than
        // twice the planes in one CTA per SM).  On small volumes (fewer
        // tiles than SMs) the output channels split into slices.
        BrickArgs br;
        br.x = static_cast<const uint4*>(x);
        br.bias = bias;
        br.y = y;
        br.out_bf16 = out_bf16 ? 1 : 0;
        br.B = B; br.D = D; br.H = H; br.W = W;
        br.cin = Cin; br.cout = Cout; br.relu = relu ? 1 : 0;
        br.kc = Cin <= CONV_KMAX ? Cin : CONV_KMAX;
        br.nch = Cin / br.kc;
        br.tiles_x = (W + 7) / 8;
        br.tiles_y = (H + 15) / 16;
        br.P = 1;
        br.nbuf = 3;
        br.ns = Cout;
        // with 16 input channels (a small brick) and at most 32 output
        // channels, two planes per CTA and twice the CTAs per SM hide the
        // staging latency better (measured 5-7% faster; wider layers lose)
        const int col_cap = (Cin == 16 && ncols == 32) ? 64 : 256;
        for (int p = 4; p >= 1; p >>= 1) {
            if (p * ncols > col_cap || (p > 1 && p > D)) continue;
            const size_t wst = (size_t)Cout * br.kc * 2;
            const size_t brick = (size_t)(br.kc / 8) * brick_plane_bytes(p);
            int nbf = CONV_MAXBUF;
            while (nbf > 3 && brick + nbf * wst > 110 * 1024) --nbf;
            if (brick + nbf * wst <= 110 * 1024 || p == 1) { br.P = p; br.nbuf = nbf; break; }
        }
        br.tiles_z = (D + br.P - 1) / br.P;
        long long tiles = (long long)br.tiles_x * br.tiles_y * br.tiles_z * B;
        while (br.ns % 32 == 0 && tiles * (Cout / br.ns) < sm_count) br.ns /= 2;
        br.ncols = 32;
        while (br.ncols < br.ns) br.ncols <<= 1;
        br.zs = 0;
        br.tcols = br.P * br.ncols;
        // z-stacked taps for slices of at most 64 output channels: an MMA of
        // N = 16..64 reads its 128 x 16 A operand for little work, so the
        // three dz taps of one (dy, dx) go into one MMA of N = 3 ns over each
        // brick plane, (P + 2) / (3 P) of the MMAs and A reads.  Four planes
        // per CTA (or two) whose (P + 4) ns accumulator columns fit 256 (two
        // CTAs per SM), whose brick and one weight image fit, and that still
        // give every SM a CTA; eight planes (fewer CTAs per SM) measured
        // slower on the 128^3 16->16 layer (0.122 vs 0.097 ms).
        if (br.ns <= 64) {
            for (int pz : {4, 2}) {
                if (pz > 2 && pz > D) continue;
                int tc = 32;
                while (tc < (pz + 4) * br.ns) tc <<= 1;
                const long long tz = (long long)br.tiles_x * br.tiles_y * ((D + pz - 1) / pz) * B;
                if (tc > 256 || (pz > 2 && tz * (Cout / br.ns) < sm_count)) continue;
                if ((size_t)(br.kc / 8) * brick_plane_bytes(pz) + (size_t)3 * br.ns * br.kc * 2 > 110 * 1024) continue;
                br.zs = 1;
                br.P = pz;
                br.tcols = tc;
                br.tiles_z = (D + pz - 1) / pz;
                tiles = tz;
                break;
            }
        }
        const int nimg = br.zs ? 9 : 27;  // B images per chunk
        const size_t wst = (size_t)(br.zs ? 3 : 1) * br.ns * br.kc * 2;
        const size_t brick = (size_t)(br.kc / 8) * brick_plane_bytes(br.P);
        // images per weight stage: small weight images are moved several per
        // bulk copy (fewer waits in the MMA thread's chain)
        br.tps = 1;
        for (int tp : {27, 9, 3})
            if (tp <= nimg && tp * wst <= 24 * 1024 && brick + tp * wst <= 110 * 1024) { br.tps = tp; break; }
        const int stages = br.nch * (nimg / br.tps);
        br.nbuf = stages < CONV_MAXBUF ? stages : CONV_MAXBUF;
        while (br.nbuf > 1 && brick + br.nbuf * br.tps * wst > 110 * 1024) --br.nbuf;
        // + 128: the brick is aligned to 128 bytes inside the dynamic block
        size_t smem = 128 + brick + br.nbuf * br.tps * wst + (2 * CONV_MAXBUF + 2) * sizeof(uint64_t) + 32;
        // every resident CTA's tensor-memory allocation must fit at once
        const size_t ctas = 512 / br.tcols;
        const size_t smem_min = per_sm / (ctas + 1) - 1024 + 16;
        if (smem < smem_min) smem = smem_min;
        if (tiles >= (1LL << 31) || smem > 200 * 1024) return NGF_EBOUNDS;
        if (!brick_attr_set()) return NGF_ECUDA;
        // weights repacked per (slice, chunk, tap) into the B operand's
        // shared-memory image
        void* wp = nullptr;
        if (dev_alloc(&wp, 27 * (size_t)Cout * Cin * 2, st) != cudaSuccess) return NGF_ENOMEM;
        const long long chunks = 27LL * Cout * (Cin / 8);
        const dim3 pg((unsigned)((chunks + 255) / 256));
        const cudaError_t pe =
            mirrored ? launch(k_conv3d_pack_wT, pg, dim3(256), 0, st, static_cast<const __nv_bfloat16*>(w),
                              static_cast<uint4*>(wp), (int)Cin, (int)Cout, br.ns, br.kc, br.zs)
                     : launch(k_conv3d_pack_w, pg, dim3(256), 0, st, static_cast<const uint4*>(w),
                              static_cast<uint4*>(wp), (int)Cout, (int)Cin, br.ns, br.kc, br.zs);
        CUtensorMap xmap;
        const bool mapped = brick_map(&xmap, x, B, D, H, W, Cin, br.P);
        const bool ok = pe == cudaSuccess && mapped &&
                        (br.w = static_cast<const uint4*>(wp),
                         launch(k_conv3d_brick, dim3((unsigned)tiles, (unsigned)(Cout / br.ns)), dim3(CONV_THREADS),
                                smem, st, br, xmap) == cudaSuccess);
        dev_free(wp, st);
        return ok ? NGF_OK : NGF_ECUDA;
    }
}

}  // namespace
}  // namespace ngf

extern "C" ngf_status ngf_conv3d_fwd(const void* x, const void* w, const float* bias, float* y, int32_t B,
                                     int32_t D, int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t relu,
                                     void* cuda_stream) {
    return conv_run(x, w, false, bias, y, false, B, D, H, W, Cin, Cout, relu, cuda_stream);
}

extern "C" ngf_status ngf_conv3d_fwd_ex(const void* x, const void* w, const float* bias, void* y, int32_t B,
                                        int32_t D, int32_t H, int32_t W, int32_t Cin, int32_t Cout, int32_t flags,
                                        void* cuda_stream) {
    if (flags & ~(NGF_CONV_RELU | NGF_CONV_OUT_BF16)) return NGF_EINVAL;
    return conv_run(x, w, false, bias, y, (flags & NGF_CONV_OUT_BF16) != 0, B, D, H, W, Cin, Cout,
                    (flags & NGF_CONV_RELU) != 0, cuda_stream);
}

extern "C" ngf_status ngf_conv3d_dgrad(const void* dy, const void* w, void* dx, int32_t B, int32_t D, int32_t H,
                                       int32_t W, int32_t Cin, int32_t Cout, int32_t flags, void* cuda_stream) {
    if (flags & ~NGF_CONV_OUT_BF16) return NGF_EINVAL;
    // the mirrored convolution reads Cout channels and writes Cin
    return conv_run(dy, w, true, nullptr, dx, (flags & NGF_CONV_OUT_BF16) != 0, B, D, H, W, Cout, Cin, 0,
                    cuda_stream);
}

extern "C" ngf_status ngf_conv3d_wgrad(const void* dy, const void* x, float* dw, float* db, int32_t B, int32_t D,
                                       int32_t H, int32_t W, int32_t Cin, int32_t Cout, void* cuda_stream) {
    if (B < 0 || D < 0 || H < 0 || W < 0) return NGF_EINVAL;
    if (Cin < 16 || Cin % 16 != 0 || (Cin > CONV_KMAX && Cin % CONV_KMAX != 0)) return NGF_EINVAL;
    if (Cout < 16 || Cout > 128 || Cout % 16 != 0) return NGF_EINVAL;
    const long long V = (long long)B * D * H * W;
    if (V >= (1LL << 31)) return NGF_EBOUNDS;
    if (!dy || !x || !dw) return NGF_EINVAL;
    if (((uintptr_t)dy | (uintptr_t)x | (uintptr_t)dw) & 15u) return NGF_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    if (V == 0) {
        if (cudaMemsetAsync(dw, 0, 27 * (size_t)Cout * Cin * sizeof(float), st) != cudaSuccess) return NGF_ECUDA;
        if (db && cudaMemsetAsync(db, 0, (size_t)Cout * sizeof(float), st) != cudaSuccess) return NGF_ECUDA;
        return NGF_OK;
    }
    int dev = 0, sm_count = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return NGF_ECUDA;
    WgradArgs a;
    a.x = static_cast<const uint4*>(x);
    a.dy = static_cast<const uint4*>(dy);
    a.B = B; a.D = D; a.H = H; a.W = W; a.cin = Cin; a.cout = Cout;
    a.kc = Cin <= CONV_KMAX ? Cin : CONV_KMAX;
    const int nch = Cin / a.kc;
    a.tcols = 256;  // two CTAs per SM
    a.tg = a.tcols / a.kc;
    if (a.tg > 27) a.tg = 27;
    a.ntg = (27 + a.tg - 1) / a.tg;
    a.ngroups = nch * a.ntg;
    a.gcols = a.tg * a.kc;
    // the largest tile whose operands fit about 100 KB of shared memory
    const int cand[][2] = {{8, 4}, {8, 2}, {4, 4}, {4, 2}, {2, 2}, {2, 1}, {1, 1}};
    size_t smem = 0;
    for (const auto& c : cand) {
        const int TY = c[0], TZ = c[1];
        const int lines = TY * TZ, cgo = Cout / 8, cgi = a.kc / 8;
        // dy tile, plus the rows of the 128-row A operand beyond cout (they
        // alias the next voxel groups, up to 16 channel groups past the last
        // line's start)
        const size_t ab = (size_t)2 * lines * cgo * 128 + (size_t)16 * cgo * 128 + 256;
        const size_t nbv = (size_t)(WG_TX + 2) * (TY + 2) * (TZ + 2);
        const size_t bb = (size_t)(cgi + 1) * nbv * 16;
        smem = ab + bb + 64;
        a.TY = TY; a.TZ = TZ; a.a_bytes = (uint32_t)ab;
        if (smem <= 100 * 1024) break;
    }
    // at most two resident CTAs per SM, so that both tensor-memory
    // allocations (256 columns each) always fit at once
    int smem_sm = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess)
        return NGF_ECUDA;
    const size_t smem_min = (size_t)smem_sm / 3 - 1024 + 16;
    if (smem < smem_min) smem = smem_min;
    if (smem > 200 * 1024) return NGF_EBOUNDS;
    a.tiles_x = (W + WG_TX - 1) / WG_TX;
    a.tiles_y = (H + a.TY - 1) / a.TY;
    a.tiles_z = (D + a.TZ - 1) / a.TZ;
    const long long ntiles = (long long)a.tiles_x * a.tiles_y * a.tiles_z * B;
    if (ntiles >= (1LL << 31)) return NGF_EBOUNDS;
    a.ntiles = (int)ntiles;
    long long split = (2LL * sm_count + a.ngroups - 1) / a.ngroups;
    if (split > ntiles) split = ntiles;
    if (split < 1) split = 1;
    a.split = (int)split;
    if (!wgrad_attr_set()) return NGF_ECUDA;
    void* part = nullptr;
    const size_t part_bytes = (size_t)a.split * a.ngroups * Cout * a.gcols * sizeof(float);
    if (dev_alloc(&part, part_bytes, st) != cudaSuccess) return NGF_ENOMEM;
    a.part = static_cast<float*>(part);
    const long long total = 27LL * Cout * Cin;
    bool ok = launch(k_conv3d_wgrad, dim3((unsigned)a.split, (unsigned)a.ngroups), dim3(CONV_THREADS), smem, st,
                     a) == cudaSuccess &&
              launch(k_conv3d_wgrad_reduce, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, st,
                     (const float*)a.part, dw, (int)Cout, (int)Cin, a.kc, a.tg, a.ntg, a.ngroups, a.gcols,
                     a.split) == cudaSuccess;
    dev_free(part, st);
    if (ok && db) {
        const int per_block = 2048;
        const long long nb = (V + per_block - 1) / per_block;
        void* bp = nullptr;
        if (dev_alloc(&bp, (size_t)nb * Cout * sizeof(float), st) != cudaSuccess) return NGF_ENOMEM;
        ok = launch(k_bias_grad_part, dim3((unsigned)nb), dim3(128), 0, st, static_cast<const __nv_bfloat16*>(dy),
                    static_cast<float*>(bp), V, (int)Cout, per_block) == cudaSuccess &&
             launch(k_bias_grad_sum, dim3(1), dim3(256), 0, st, (const float*)bp, db, (int)nb, (int)Cout) ==
                 cudaSuccess;
        dev_free(bp, st);
    }
    return ok ? NGF_OK : NGF_ECUDA;
}

extern "C" int32_t ngf_conv3d_check(void* cuda_stream) {
    if (cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)) != cudaSuccess) return NGF_ECUDA;
    unsigned int n = 0;
    if (cudaMemcpyFromSymbol(&n, g_conv_timeouts, sizeof(n)) != cudaSuccess) return NGF_ECUDA;
    const unsigned int zero = 0;
    if (cudaMemcpyToSymbol(g_conv_timeouts, &zero, sizeof(zero)) != cudaSuccess) return NGF_ECUDA;
    return (int32_t)n;
}
