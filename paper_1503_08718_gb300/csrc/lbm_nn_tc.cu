// 3x3x3 convolution of the warm-start network on the fifth-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory), sm_103a.
//
// Implicit GEMM: M = output voxels, N = output channels, K = 27 taps x input
// channels.  A tile is 128 output voxels (16 rows of 8 voxels of one z plane
// of one cell) for all output channels, times tz consecutive planes.  Instead
// of gathering an im2col matrix per tap, the tile's halo is staged once in
// shared memory: tz + 2 planes x 18 rows x 10 voxels of 16-byte channel
// chunks, laid out so that every tap's A operand is the same canonical
// no-swizzle K-major layout (8-row core matrices of 16-byte rows) at a
// different start address: rows of 8 voxels are 16 bytes apart, the 16 rows
// of the tile 160 bytes apart (SBO) and consecutive 8-channel chunks one halo
// plane set apart (LBO).  The 27 taps then cost 27 x K/16 MMA instructions
// and no extra copies.  The B operand (the tap's weights, K-major
// [cout][cin]) streams through a ring of shared-memory stages; tcgen05.commit
// on per-stage mbarriers frees each stage when the MMAs that read it are
// done.  The forward kernel is persistent with warp roles (weight producer,
// MMA issuer, halo loaders, epilogue) and two accumulator buffers in tensor
// memory, so that loads, MMAs and the epilogue of consecutive tiles overlap.
// Padding as the rest of the network: periodic in x and y, zero in z.
//
// Every wait on an mbarrier is bounded: on expiry the kernel records an
// error word (read by lbm_nn_tc_error), waits (bounded again) for the MMAs
// it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <algorithm>
#include <type_traits>

#include "lbm.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int TILE_Y = 16, TILE_X = 8;             // 128 output voxels per block
constexpr int HY = TILE_Y + 2, HX = TILE_X + 2;     // halo of a tile's plane
constexpr int THREADS = 128;
constexpr unsigned kSpinLimit = 1u << 22;          // bounded mbarrier waits

__device__ unsigned int g_tc_error = 0u;           // first error code of any block

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared; src_bytes 0 fills zeros
__device__ __forceinline__ void cp16(unsigned dst, const void* src, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Waits until the mbarrier's phase `parity` has completed; false on timeout.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    for (unsigned i = 0; i < kSpinLimit; ++i) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading
// (K-direction core matrix) and stride (8-row group) byte offsets, the fixed
// version bits 46..48 = 0b001, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
    unsigned r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct Vol {
    int n, d, h, w;
};

// Input channels per shared-memory halo (a channel group): 32 where they
// divide the input channels, else 16.
__host__ __device__ constexpr int cg_for(int cin) {
    return cin % 32 == 0 ? 32 : 16;
}

// Forward kernel: persistent blocks (one per SM) with warp roles, each block
// walking the tiles blockIdx.x, blockIdx.x + gridDim.x, ...  A tile is TZ
// consecutive z planes of the same 16 x 8 rows (TZ accumulators of N columns
// that share every weight slab).
//   warp 0 (one thread): streams the weight slabs, tile after tile, through
//     a ring of WS stages (cp.async.bulk, completion on the stage's `w_full`
//     mbarrier, the stage freed by the MMAs' commit to `w_empty`);
//   warp 1 (one thread): issues the MMAs of each (tap, channel group) as its
//     slab and halo are in, into one of two accumulator buffers (tile k uses
//     buffer k & 1), and commits the halo stage to `h_empty` and the finished
//     tile to `a_full`;
//   warps 2-5: load each (tile, channel group) halo into a ring of HS stages
//     (cp.async, zero fill outside the cell in z), then fence it for the
//     tensor core and arrive on `h_full`;
//   warps 6-9: the epilogue of tile k (tcgen05.ld of its buffer, bias, leaky
//     ReLU, store) while the MMAs of tile k + 1 run in the other buffer; they
//     free the buffer on `a_empty`.
// The weights arrive pre-arranged (lbm_nn_weights_kmajor): slab (tap, group)
// is [cg/8][N][8] BF16, exactly the stage's shared-memory image.
constexpr int W_LOAD = 2, N_LOAD = 4, W_EPI = 6;   // first loader warp, loader warps, first epilogue warp
constexpr int PT = 32 * (W_EPI + 4);               // threads of the forward kernel

__host__ __device__ constexpr size_t tc_halo_bytes(int cg, int tz) { return (size_t)(tz + 2) * HY * HX * cg * 2; }
__host__ __device__ constexpr size_t tc_smem_bytes(int cg, int n, int tz, int ws, int hs) {
    return (size_t)hs * tc_halo_bytes(cg, tz) + (size_t)ws * n * cg * 2 + 8 * (2 * ws + 2 * hs + 5) + 16;
}

// Blocks an SM can hold are bounded by shared memory; make sure they never
// ask for more than the SM's 512 tensor-memory columns together (a block
// whose tcgen05.alloc cannot be served waits for another to free).
size_t tmem_safe_smem(size_t smem, int cols) {
    const int max_blocks = 512 / cols;
    const size_t floor = (size_t)(227 * 1024) / (size_t)(max_blocks + 1) + 1;
    return smem > floor ? smem : floor;
}

// waits of a whole warp that is not on the critical path: every lane polls
// with a short sleep between polls (so that the spinning warps leave the
// issue slots to the MMA thread); the outcome is the warp's
__device__ __forceinline__ bool warp_wait(unsigned bar, unsigned parity) {
    bool ok = false;
    for (unsigned i = 0; i < kSpinLimit && !ok; ++i) {
        unsigned r;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(r)
            : "r"(bar), "r"(parity)
            : "memory");
        ok = r != 0;
        if (!ok) __nanosleep(64);
    }
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void mbar_arrive(unsigned bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <bool RELU, bool OUT_F32, int TZ>
__global__ void __launch_bounds__(PT, 1) conv3_tc_kernel(const bf16* __restrict__ X, int Cin, int CG,
                                                         const bf16* __restrict__ Wu,
                                                         const float* __restrict__ bias,
                                                         void* __restrict__ Yv, int N, int tstride,
                                                         int tmem_cols, Vol vol, int n_tiles, int WS, int HS) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CG8 = CG >> 3;
    constexpr int PZ = TZ + 2;                      // halo planes
    constexpr int PVOX = PZ * HY * HX;              // halo voxels
    const unsigned hstage = (unsigned)PVOX * CG * 2;
    const unsigned slab = (unsigned)N * CG * 2;     // bytes of one weight slab
    unsigned char* halo = smem;
    unsigned char* wst = smem + (size_t)HS * hstage;
    unsigned long long* w_full = reinterpret_cast<unsigned long long*>(wst + (size_t)WS * slab);
    unsigned long long* w_empty = w_full + WS;
    unsigned long long* h_full = w_empty + WS;
    unsigned long long* h_empty = h_full + HS;
    unsigned long long* a_full = h_empty + HS;      // [2]
    unsigned long long* a_empty = a_full + 2;       // [2]
    unsigned long long* done = a_empty + 2;
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(done + 1);
    __shared__ volatile int s_fail;
    __shared__ long long s_issued, s_consumed;      // weight slabs issued / waited for
    const unsigned halo_s = smem_u32(halo), wst_s = smem_u32(wst);
    const int ngroups = Cin / CG;
    const int per_tile = 27 * ngroups;              // weight slabs per tile, group-major
    const int tiles_x = vol.w / TILE_X, tiles_y = vol.h / TILE_Y, zt = vol.d / TZ;
    const int my_tiles = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (tid == 0) {
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        for (int s = 0; s < WS; ++s) {
            mbar_init(smem_u32(&w_full[s]), 1);
            mbar_init(smem_u32(&w_empty[s]), 1);
        }
        for (int s = 0; s < HS; ++s) {
            mbar_init(smem_u32(&h_full[s]), 32 * N_LOAD);
            mbar_init(smem_u32(&h_empty[s]), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&a_full[s]), 1);
            mbar_init(smem_u32(&a_empty[s]), 128);
        }
        mbar_init(smem_u32(done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = *tmem_slot;

    // cell, first plane, first row and first voxel of this block's tile k
    auto tile_at = [&](int k, int& n0, int& z0, int& y0, int& x0) {
        int b = (int)blockIdx.x + k * (int)gridDim.x;
        const int tx = b % tiles_x; b /= tiles_x;
        const int ty = b % tiles_y; b /= tiles_y;
        z0 = (b % zt) * TZ;
        n0 = b / zt;
        x0 = tx * TILE_X;
        y0 = ty * TILE_Y;
    };

    if (warp == 0) {
        if (lane == 0) {                            // weight producer
            const long long total = (long long)my_tiles * per_tile;
            long long T = 0;
            int s = 0, g = 0, t = 0;                // stage, channel group, tap of slab T
            unsigned round = 0;                     // fills of stage s so far
            for (; T < total && !s_fail; ++T) {
                if (round > 0 && !mbar_wait(smem_u32(&w_empty[s]), (round - 1) & 1u)) {
                    s_fail = 1;
                    break;
                }
                const unsigned fb = smem_u32(&w_full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(slab)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        wst_s + (unsigned)s * slab),
                    "l"(Wu + (size_t)(t * ngroups + g) * (slab / 2)), "r"(slab), "r"(fb)
                    : "memory");
                if (++s == WS) {
                    s = 0;
                    ++round;
                }
                if (++t == 27) {
                    t = 0;
                    if (++g == ngroups) g = 0;
                }
            }
            s_issued = T;
        }
    } else if (warp == 1) {
        if (lane == 0) {                            // MMA issuer
            const uint32_t idesc = instr_desc(N);
            const unsigned lbo_a = PVOX * 16, sbo_a = HX * 16;
            const unsigned lbo_b = (unsigned)N * 16, sbo_b = 128;
            // descriptors of halo stage 0 and weight stage 0; a start address
            // is the descriptor's low field in 16-byte units, so an offset
            // within shared memory is added to it directly
            const uint64_t ad0 = smem_desc(halo_s, lbo_a, sbo_a);
            const uint64_t bd0 = smem_desc(wst_s, lbo_b, sbo_b);
            long long T = 0;
            int ws = 0, hs = 0;                     // weight and halo stage
            unsigned wround = 0, hround = 0;        // completed passes over each ring
            for (int k = 0; k < my_tiles && !s_fail; ++k) {
                const int ab = k & 1;
                if (k >= 2 && !mbar_wait(smem_u32(&a_empty[ab]), (unsigned)(((k >> 1) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                fence_after();
                const unsigned dacc = tmem + (unsigned)(ab * TZ * tstride);
                for (int g = 0; g < ngroups && !s_fail; ++g) {
                    if (!mbar_wait(smem_u32(&h_full[hs]), hround & 1u)) {
                        s_fail = 1;
                        break;
                    }
                    const uint64_t adh = ad0 + (uint64_t)((hs * hstage) >> 4);
                    for (int t = 0; t < 27; ++t, ++T) {
                        if (!mbar_wait(smem_u32(&w_full[ws]), wround & 1u)) {
                            s_fail = 1;
                            break;
                        }
                        s_consumed = T + 1;
                        fence_after();
                        const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                        const uint64_t bdw = bd0 + (uint64_t)((ws * slab) >> 4);
                        // consecutive MMAs go to different accumulators: MMAs into
                        // one accumulator follow each other only after the
                        // previous one is done
                        for (int ks = 0; ks < CG / 16; ++ks)
#pragma unroll
                            for (int tz = 0; tz < TZ; ++tz) {
                                const uint64_t ad = adh + (uint64_t)((((tz + dz) * HY + dy) * HX + dx));
                                mma_bf16(dacc + (unsigned)(tz * tstride), ad + (uint64_t)(ks * (2 * lbo_a >> 4)),
                                         bdw + (uint64_t)(ks * (2 * lbo_b >> 4)), idesc,
                                         (g > 0 || t > 0 || ks > 0) ? 1u : 0u);
                            }
                        mma_commit(smem_u32(&w_empty[ws]));
                        if (++ws == WS) {
                            ws = 0;
                            ++wround;
                        }
                    }
                    if (s_fail) break;
                    mma_commit(smem_u32(&h_empty[hs]));
                    if (++hs == HS) {
                        hs = 0;
                        ++hround;
                    }
                }
                if (s_fail) break;
                mma_commit(smem_u32(&a_full[ab]));
            }
            // every MMA issued is done before the block frees its tensor memory
            mma_commit(smem_u32(done));
            if (!mbar_wait(smem_u32(done), 0u)) s_fail = 1;
        }
    } else if (warp < W_EPI) {                      // halo loaders
        // thread lt owns cell j = lt % rc of every rc-cell halo row (a row:
        // HX voxels x CG/8 chunks) and walks rows r0, r0 + rs, ...
        const int lt = tid - 32 * W_LOAD;
        const int rc = HX * CG8, rs = (32 * N_LOAD) / rc;
        const int j = lt % rc, r0 = lt / rc;
        const int xh = j / CG8, c8 = j - xh * CG8;
        int hs = 0;                                 // halo stage
        unsigned hround = 0;                        // completed passes over the ring
        for (int k = 0; k < my_tiles && !s_fail; ++k) {
            int n0, z0, y0, x0;
            tile_at(k, n0, z0, y0, x0);
            int x = x0 + xh - 1;
            x = x < 0 ? x + vol.w : (x >= vol.w ? x - vol.w : x);
            for (int g = 0; g < ngroups; ++g) {
                if (hround > 0 && !warp_wait(smem_u32(&h_empty[hs]), (hround - 1) & 1u)) {
                    s_fail = 1;
                    break;
                }
                const unsigned hb = halo_s + (unsigned)hs * hstage + (unsigned)(((c8 * PZ) * HY * HX + xh) * 16);
                const bf16* xs = X + (long long)x * Cin + g * CG + c8 * 8;
                if (r0 < rs)
                    for (int row = r0; row < PZ * HY; row += rs) {
                        const int zz = row / HY, yh = row - zz * HY;
                        const int z = z0 + zz - 1;
                        int y = y0 + yh - 1;
                        y = y < 0 ? y + vol.h : (y >= vol.h ? y - vol.h : y);
                        const bool in = z >= 0 && z < vol.d;
                        const long long rowv = (((long long)n0 * vol.d + (in ? z : 0)) * vol.h + y) * vol.w;
                        cp16(hb + (unsigned)(row * HX * 16), xs + rowv * Cin, in ? 16u : 0u);
                    }
                cp_commit();
                cp_wait_all();
                fence_proxy_async();                // the tensor core reads it through the async proxy
                mbar_arrive(smem_u32(&h_full[hs]));
                if (++hs == HS) {
                    hs = 0;
                    ++hround;
                }
            }
        }
    } else {                                        // epilogue
        const int q = warp & 3;                     // TMEM lanes 32q .. 32q + 31 (warps 6-9: 2, 3, 0, 1)
        const int m = q * 32 + lane;                // output voxel m of the tile's planes
        const int yy = m / TILE_X, xx = m % TILE_X;
        for (int k = 0; k < my_tiles && !s_fail; ++k) {
            const int ab = k & 1;
            if (!warp_wait(smem_u32(&a_full[ab]), (unsigned)((k >> 1) & 1))) {
                s_fail = 1;
                break;
            }
            fence_after();
            int n0, z0, y0, x0;
            tile_at(k, n0, z0, y0, x0);
            for (int tz = 0; tz < TZ; ++tz)
                for (int c0 = 0; c0 < N; c0 += 16) {
                    const long long v = (((long long)n0 * vol.d + z0 + tz) * vol.h + y0 + yy) * vol.w + x0 + xx;
                    const unsigned trow = tmem + ((unsigned)(q * 32) << 16) + (unsigned)((ab * TZ + tz) * tstride);
                    float acc[16];
                    tmem_ld16(trow + (unsigned)c0, acc);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float y = acc[i] + (bias ? bias[c0 + i] : 0.f);
                        if (RELU) y = y > 0.f ? y : 0.01f * y;
                        acc[i] = y;
                    }
                    if (OUT_F32) {
                        float4* dst = reinterpret_cast<float4*>(reinterpret_cast<float*>(Yv) + v * N + c0);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            dst[u] = make_float4(acc[4 * u], acc[4 * u + 1], acc[4 * u + 2], acc[4 * u + 3]);
                    } else {
                        __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) o[u] = __floats2bfloat162_rn(acc[2 * u], acc[2 * u + 1]);
                        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(Yv) + v * N + c0);
                        dst[0] = *reinterpret_cast<const uint4*>(&o[0]);
                        dst[1] = *reinterpret_cast<const uint4*>(&o[4]);
                    }
                }
            fence_before();
            mbar_arrive(smem_u32(&a_empty[ab]));
        }
    }
    __syncthreads();
    // after a failure, the weight copies still in flight land before the
    // block leaves (bounded waits on the last phase of each stage)
    if (tid == 0 && s_fail)
        for (long long T = s_consumed; T < s_issued; ++T)
            mbar_wait(smem_u32(&w_full[T % WS]), (unsigned)((T / WS) & 1));
    if (tid == 0 && s_fail) atomicCAS(&g_tc_error, 0u, 1u);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores: dW[tap][ci][co] = sum_v X[v + tap][ci]
// G[v][co].  Per tap a GEMM D[co][ci] (M = output channels, zero-padded to
// 128; N = a group of at most 64 input channels; K = voxels).  Both operands
// are channels-last in memory, so both enter the MMA MN-major: 16-byte rows
// of 8 channels, one per voxel.  A block owns one column of 16 x 8 tiles
// (cell n0, rows y0..y0+15, voxels x0..x0+7) over a range of planes, a group
// of taps and a group of CG input channels, and keeps one accumulator per tap
// in tensor memory (512 columns: 8 taps of 64 channels, 16 of 32, 27 of 16);
// each tap's B operand is the input halo seen through its own descriptor.
// The halo lives in a ring of four planes ([CG/8][4 slots][18][10] x 16 B):
// tile z reads planes z-1, z, z+1 and, while its MMAs run, the block loads
// plane z+2 into the fourth slot together with the next output-gradient tile
// (two G buffers), so each tile brings in one halo plane, not three.  Each G
// buffer has its own mbarrier (tile k commits to bar[k & 1]), so a wait never
// lags its barrier by more than one phase.  At the end the accumulators are
// added into dW (FP32 atomics, dW zeroed by the caller).
// MN-major no-swizzle layout: core matrices of 8 K-rows x 16 bytes; the
// descriptor's LBO is the stride between core matrices along K and its SBO
// the stride along M (N).
constexpr int WGZ_TMEM = 512;

template <int CG>
__global__ void __launch_bounds__(THREADS) conv3_wgrad_z_kernel(const bf16* __restrict__ X, int Cin,
                                                                const bf16* __restrict__ G, int Cout,
                                                                float* __restrict__ dW, Vol vol, int zchunk,
                                                                int groups_per_block, int ns) {
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int CG8 = CG / 8;
    constexpr int RING = 4;                        // a power of two
    constexpr int PLANE = HY * HX;                 // halo voxels of one plane
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* ring = smem;                    // [CG/8][4][18][10] x 16 B
    unsigned char* gs = ring + (size_t)RING * PLANE * CG * 2;   // 2 x [16][128] x 16 B
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(gs + 2 * 16 * 128 * 16);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar + 2);
    __shared__ volatile int s_fail;
    const unsigned ring_s = smem_u32(ring), gs_s = smem_u32(gs);
    const int Cout8 = Cout / 8;
    // MMA groups: per (dz, dy) the taps dx = dxb .. dxb + ns - 1 with dxb =
    // 0, ns, ..; ceil(3 / ns) groups per (dz, dy)
    const int gpd = (3 + ns - 1) / ns;
    const int q0 = blockIdx.y * groups_per_block;
    const int nq = min(groups_per_block, 9 * gpd - q0);
    const int g = blockIdx.z;
    // per group of this block: dz and the tap's start within a halo plane
    // (dy HX + dx), computed once (no divisions in the MMA thread's loop)
    __shared__ int s_gdz[32], s_goff[32];
    for (int j = threadIdx.x; j < nq; j += THREADS) {
        const int q = q0 + j, dzdy = q / gpd;
        s_gdz[j] = dzdy / 3;
        s_goff[j] = (dzdy % 3) * HX + (q % gpd) * ns;
    }

    const int tiles_x = vol.w / TILE_X, tiles_y = vol.h / TILE_Y;
    const int zchunks = (vol.d + zchunk - 1) / zchunk;
    int b = blockIdx.x;
    const int zc = b % zchunks; b /= zchunks;
    const int tx = b % tiles_x; b /= tiles_x;
    const int ty = b % tiles_y; b /= tiles_y;
    const int n0 = b;
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y;
    const int zb = zc * zchunk, ze = min(zb + zchunk, vol.d);

    // the rows past the ns shifted copies of G (ns * Cout .. 127) stay zero in both buffers
    const int used8 = ns * Cout8;
    for (int i = tid; i < 2 * (16 - used8) * 128; i += THREADS) {
        const int buf = i / ((16 - used8) * 128), r = i % ((16 - used8) * 128);
        *reinterpret_cast<uint4*>(gs + (size_t)buf * 16 * 128 * 16 + (size_t)(used8 * 128 + r) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid == 0) {
        s_fail = 0;
        mbar_init(smem_u32(&bar[0]), 1);
        mbar_init(smem_u32(&bar[1]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(WGZ_TMEM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const unsigned tmem = *tmem_slot;
    const uint32_t idesc = instr_desc(CG) | (1u << 15) | (1u << 16);   // both operands MN-major

    // halo plane z (any z; outside the cell: zeros) into its ring slot
    auto load_plane = [&](int z) {
        const int slot = (z + RING) % RING;
        const bool in = z >= 0 && z < vol.d;
        for (int i = tid; i < PLANE * CG8; i += THREADS) {
            const int hv = i / CG8, c8 = i - hv * CG8;
            const int xh = hv % HX, yh = hv / HX;
            int y = y0 + yh - 1, x = x0 + xh - 1;
            y = y < 0 ? y + vol.h : (y >= vol.h ? y - vol.h : y);
            x = x < 0 ? x + vol.w : (x >= vol.w ? x - vol.w : x);
            const long long v = (((long long)n0 * vol.d + (in ? z : 0)) * vol.h + y) * vol.w + x;
            cp16(ring_s + (unsigned)((((c8 * RING + slot) * HY + yh) * HX + xh) * 16),
                 X + v * Cin + g * CG + c8 * 8, in ? 16u : 0u);
        }
    };
    // copy s of the output-gradient tile (rows s * Cout .. s * Cout + Cout - 1)
    // holds G at x - s: with the halo of tap (dz, dy, dxb) it gives tap
    // (dz, dy, dxb + s), because sum_v G[v - s] X[v + t] = sum_u G[u] X[u + s + t]
    // over the periodic rows
    auto load_g = [&](int z, int buf) {
        if (ns == 1) {                             // one copy: no shift
            for (int i = tid; i < 128 * Cout8; i += THREADS) {
                const int v = i / Cout8, c8 = i - v * Cout8;
                const long long gv =
                    (((long long)n0 * vol.d + z) * vol.h + y0 + v / TILE_X) * vol.w + x0 + v % TILE_X;
                cp16(gs_s + (unsigned)(buf * 16 * 128 * 16 + (c8 * 128 + v) * 16), G + gv * Cout + c8 * 8, 16u);
            }
            return;
        }
        for (int i = tid; i < 128 * used8; i += THREADS) {
            const int v = i / used8, r8 = i - v * used8;
            const int sft = r8 / Cout8, c8 = r8 - sft * Cout8;
            int x = x0 + v % TILE_X - sft;
            x = x < 0 ? x + vol.w : x;
            const long long gv = (((long long)n0 * vol.d + z) * vol.h + y0 + v / TILE_X) * vol.w + x;
            cp16(gs_s + (unsigned)(buf * 16 * 128 * 16 + (r8 * 128 + v) * 16), G + gv * Cout + c8 * 8, 16u);
        }
    };
    auto wait_tile = [&](int k) {                  // thread 0: tile k's MMAs are done
        if (tid == 0 && !s_fail && !mbar_wait(smem_u32(&bar[k & 1]), (unsigned)((k >> 1) & 1))) s_fail = 1;
    };

    const int ntiles = ze - zb;
    load_plane(zb - 1);
    load_plane(zb);
    load_plane(zb + 1);
    load_g(zb, 0);
    cp_commit();
    int issued = 0;
    for (int k = 0; k < ntiles; ++k) {
        const int z = zb + k;
        cp_wait_all();
        fence_proxy_async();
        __syncthreads();
        if (s_fail) break;
        if (tid == 0) {
            fence_after();
            const unsigned gbuf = gs_s + (unsigned)((k & 1) * 16 * 128 * 16);
            for (int j = 0; j < nq; ++j) {
                const int slot = (z + s_gdz[j] + RING - 1) & (RING - 1), off = s_goff[j];
                for (int ks = 0; ks < 128 / 16; ++ks) {
                    // A: output gradient [co][voxels] (LBO = K step of 8 voxels, SBO = 8 channels)
                    const uint64_t ad = smem_desc(gbuf + 2u * ks * 128u, 128u, 128u * 16u);
                    // B: halo [ci][voxels] of the tap (LBO = next voxel row, SBO = next 8 channels)
                    const uint64_t bd = smem_desc(
                        ring_s + (unsigned)((slot * PLANE + off + 2 * ks * HX) * 16), HX * 16,
                        RING * PLANE * 16);
                    mma_bf16(tmem + (unsigned)(j * CG), ad, bd, idesc, (k > 0 || ks > 0) ? 1u : 0u);
                }
            }
            mma_commit(smem_u32(&bar[k & 1]));
        }
        issued = k + 1;
        if (k + 1 < ntiles) {
            // plane z + 2 replaces plane z - 2 and G buffer (k + 1) & 1 held
            // tile k - 1: both wait for tile k - 1's MMAs
            if (k >= 1) wait_tile(k - 1);
            __syncthreads();
            if (s_fail) break;
            load_plane(z + 2);
            load_g(z + 1, (k + 1) & 1);
            cp_commit();
        }
    }
    cp_wait_all();
    if (issued > 0) {
        wait_tile(issued - 1);
        if (tid == 0 && s_fail) mbar_wait(smem_u32(&bar[(issued - 1) & 1]), (unsigned)(((issued - 1) >> 1) & 1));
    }
    __syncthreads();
    fence_after();
    if (s_fail) {
        if (tid == 0) atomicCAS(&g_tc_error, 0u, 1u);
    } else if (issued > 0) {
        // lane l = copy l / Cout, output channel l % Cout (warp w: lanes
        // 32w .. 32w + 31), columns = ci
        const int l = warp * 32 + lane;
        const int sft = l / Cout, co = l - sft * Cout;
        const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
        for (int j = 0; j < nq; ++j) {
            const int q = q0 + j, dzdy = q / gpd;
            const int dx = (q % gpd) * ns + sft;
            const int t = dzdy * 3 + dx;
            for (int c0 = 0; c0 < CG; c0 += 16) {
                float acc[16];
                tmem_ld16(trow + (unsigned)(j * CG + c0), acc);
                if (sft < ns && dx < 3) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        atomicAdd(dW + ((long long)t * Cin + g * CG + c0 + i) * Cout + co, acc[i]);
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(WGZ_TMEM)
                     : "memory");
}

__host__ __device__ constexpr size_t wgz_smem_bytes(int cg) {
    return (size_t)4 * HY * HX * cg * 2 + (size_t)2 * 16 * 128 * 16 + 64;
}

// Weight slabs for the forward kernel from W [27][cin][cout].  The conv that
// uses them has input channels K and output channels N: K = cin, N = cout
// for the forward conv (flip 0); K = cout, N = cin with the taps reversed for
// the data gradient's conv (flip 1).  Slab (tap, group g) holds the group's
// CG = cg_for(K) input channels as [CG/8][N][8]: element
// (k8, n, e) = weight of input channel g CG + 8 k8 + e, output channel n.
__global__ void kmajor_kernel(const bf16* __restrict__ W, bf16* __restrict__ Wu, int Cin, int Cout,
                              int flip) {
    const int K = flip ? Cout : Cin, N = flip ? Cin : Cout;
    const int CG = cg_for(K), G = K / CG;
    const long long total = 27LL * K * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i & 7);
        long long r = i >> 3;
        const int n = (int)(r % N); r /= N;
        const int k8 = (int)(r % (CG / 8)); r /= CG / 8;
        const int g = (int)(r % G);
        const int tap = (int)(r / G);
        const int k = g * CG + 8 * k8 + e;                 // input channel of the conv
        Wu[i] = flip ? W[((long long)(26 - tap) * Cin + n) * Cout + k]
                     : W[((long long)tap * Cin + k) * Cout + n];
    }
}

int tmem_cols_for(int n) {
    int c = 32;
    while (c < n) c <<= 1;
    return c;
}

// Launch configuration of the forward kernel: z planes per tile (tz: the
// planes share every weight slab and give the MMA thread tz independent
// accumulators to interleave), weight stages (ws), halo stages (hs, two: one
// loading while the MMAs read the other) and persistent blocks per SM
// (per_sm: blocks on one SM interleave their MMA streams too).  The blocks
// of an SM must fit its 512 tensor-memory columns with both accumulator
// buffers each.  Default (measured on the network's layer shapes): two
// blocks per SM where tensor and shared memory hold them with at least four
// weight stages each, else one; within that the most planes per tile; as
// many weight stages as fit, up to 16.
struct TcCfg {
    int tz, ws, hs, cols, per_sm;
    size_t smem;
};

constexpr size_t kTcSmemMax = (size_t)226 * 1024;

TcCfg tc_cfg(int cin, int cout, int d, int tz_req, int ws_req) {
    const int cg = cg_for(cin);
    const int tcols = tmem_cols_for(cout);
    const int hs = 2;
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
        const size_t cap = kTcSmemMax / per_sm - (per_sm > 1 ? 1024 : 0);
        for (int tz : {4, 2, 1}) {
            if (tz_req && tz != tz_req) continue;
            if (d % tz || 2 * tz * tcols > 512) continue;
            const int cols = tmem_cols_for(2 * tz * tcols);
            if (per_sm * cols > 512) continue;
            int ws = 0;
            if (ws_req) {
                if (ws_req >= 2 && tc_smem_bytes(cg, cout, tz, ws_req, hs) <= cap) ws = ws_req;
            } else {
                for (int w = 16; w >= (per_sm > 1 ? 4 : 2) && !ws; --w)
                    if (tc_smem_bytes(cg, cout, tz, w, hs) <= cap) ws = w;
            }
            if (ws) return TcCfg{tz, ws, hs, cols, per_sm, tc_smem_bytes(cg, cout, tz, ws, hs)};
        }
    }
    return TcCfg{0, 0, 0, 0, 0, 0};
}

}  // namespace

extern "C" {

int lbm_nn_conv3d_tc_supported(int cin, int cout, int n, int d, int h, int w) {
    if (cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256) return 0;
    if (n < 1 || d < 1 || h < TILE_Y || w < TILE_X || h % TILE_Y || w % TILE_X) return 0;
    if ((long long)n * d * h * w >= (1LL << 40)) return 0;
    return tc_cfg(cin, cout, d, 0, 0).tz ? 1 : 0;
}

lbm_status lbm_nn_conv3d_tc_cfg(const void* x, int cin, const void* wk, const float* bias, void* y, int cout,
                                int n, int d, int h, int wdt, int relu, int out_f32, int tz, int ns, void* stream) {
    if (!x || !wk || !y || !lbm_nn_conv3d_tc_supported(cin, cout, n, d, h, wdt)) return LBM_ERR_INVALID_ARG;
    const TcCfg cf = tc_cfg(cin, cout, d, tz, ns);
    if (!cf.tz) return LBM_ERR_INVALID_ARG;
    const int cg = cg_for(cin);
    // at most per_sm blocks on an SM (their accumulators fill its tensor memory)
    const size_t smem = std::max(cf.smem, (size_t)(227 * 1024) / (size_t)(cf.per_sm + 1) + 1);
    const Vol vol{n, d, h, wdt};
    const long long tiles = (long long)(wdt / TILE_X) * (h / TILE_Y) * (d / cf.tz) * n;
    if (tiles > 0x7fffffffLL) return LBM_ERR_INVALID_ARG;
    int dev = 0, n_sm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)n_sm * cf.per_sm);
    cudaStream_t st = (cudaStream_t)stream;
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* W = static_cast<const bf16*>(wk);
    const int tstride = tmem_cols_for(cout);          // accumulator columns per plane
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            kern<<<grid, PT, smem, st>>>(X, cin, cg, W, bias, y, cout, tstride, cf.cols, vol, (int)tiles, cf.ws, cf.hs);
    };
    auto pick = [&](auto tzc) {
        constexpr int TZ = decltype(tzc)::value;
        if (relu && !out_f32) go(conv3_tc_kernel<true, false, TZ>);
        else if (!relu && !out_f32) go(conv3_tc_kernel<false, false, TZ>);
        else if (relu) go(conv3_tc_kernel<true, true, TZ>);
        else go(conv3_tc_kernel<false, true, TZ>);
    };
    if (cf.tz == 4) pick(std::integral_constant<int, 4>{});
    else if (cf.tz == 2) pick(std::integral_constant<int, 2>{});
    else pick(std::integral_constant<int, 1>{});
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_nn_conv3d_tc(const void* x, int cin, const void* wk, const float* bias, void* y, int cout,
                            int n, int d, int h, int wdt, int relu, int out_f32, void* stream) {
    return lbm_nn_conv3d_tc_cfg(x, cin, wk, bias, y, cout, n, d, h, wdt, relu, out_f32, 0, 0, stream);
}

int lbm_nn_conv3d_wgrad_tc_supported(int cin, int cout, int n, int d, int h, int w) {
    if (cin < 16 || cin % 16 || cout < 8 || cout % 8 || cout > 128) return 0;
    if (n < 1 || d < 1 || h < TILE_Y || w < TILE_X || h % TILE_Y || w % TILE_X) return 0;
    return (long long)n * d * h * w < (1LL << 40) ? 1 : 0;
}

lbm_status lbm_nn_conv3d_wgrad_tc(const void* x, int cin, const void* g, int cout, float* dw, int n, int d,
                                  int h, int wdt, void* stream) {
    if (!x || !g || !dw || !lbm_nn_conv3d_wgrad_tc_supported(cin, cout, n, d, h, wdt)) return LBM_ERR_INVALID_ARG;
    const int cg = cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16);
    const Vol vol{n, d, h, wdt};
    // shifted copies of the output gradient that fill the M = 128 rows: three
    // taps per MMA while 3 * cout <= 128, two while 2 * cout <= 128
    const int ns = 3 * cout <= 128 ? 3 : (2 * cout <= 128 ? 2 : 1);
    const int total = 9 * ((3 + ns - 1) / ns);           // MMA groups
    // as many groups per block as the 512 tensor-memory columns hold (a
    // balanced split measured up to 9 % slower at 128 output channels)
    const int groups_per_block = std::min(total, WGZ_TMEM / cg);
    const int tap_groups = (total + groups_per_block - 1) / groups_per_block;
    const int ci_groups = cin / cg;
    int n_sm = 152;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, 0);
    // columns of tiles; z split into chunks until there are about two waves
    // of blocks (one block per SM: all 512 TMEM columns)
    const long long columns = (long long)(wdt / TILE_X) * (h / TILE_Y) * n;
    const long long per_z = columns * tap_groups * ci_groups;
    int zchunk = d;
    while (zchunk > 4 && per_z * ((d + zchunk - 1) / zchunk) < 2LL * n_sm) zchunk = (zchunk + 1) / 2;
    const long long gx = columns * ((d + zchunk - 1) / zchunk);
    if (gx > 0x7fffffffLL) return LBM_ERR_INVALID_ARG;
    const dim3 grid((unsigned)gx, (unsigned)tap_groups, (unsigned)ci_groups);
    const size_t smem = tmem_safe_smem(wgz_smem_bytes(cg), WGZ_TMEM);
    cudaStream_t st = (cudaStream_t)stream;
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* G = static_cast<const bf16*>(g);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<grid, THREADS, smem, st>>>(X, cin, G, cout, dw, vol, zchunk, groups_per_block, ns);
    };
    if (cg == 64) go(conv3_wgrad_z_kernel<64>);
    else if (cg == 32) go(conv3_wgrad_z_kernel<32>);
    else go(conv3_wgrad_z_kernel<16>);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_nn_weights_kmajor(const void* w, void* wk, int cin, int cout, int flip, void* stream) {
    if (!w || !wk || cin < 1 || cout < 1) return LBM_ERR_INVALID_ARG;
    long long g = (27LL * cin * cout + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    kmajor_kernel<<<(int)g, 256, 0, (cudaStream_t)stream>>>(static_cast<const bf16*>(w), static_cast<bf16*>(wk),
                                                             cin, cout, flip ? 1 : 0);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

lbm_status lbm_nn_tc_error(int* out, int clear) {
    if (!out) return LBM_ERR_INVALID_ARG;
    unsigned v = 0;
    if (cudaMemcpyFromSymbol(&v, g_tc_error, sizeof v) != cudaSuccess) return LBM_ERR_CUDA;
    *out = (int)v;
    if (clear) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(g_tc_error, &z, sizeof z) != cudaSuccess) return LBM_ERR_CUDA;
    }
    return LBM_OK;
}

}  // extern "C"
