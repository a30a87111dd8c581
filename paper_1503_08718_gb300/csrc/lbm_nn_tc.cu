// 3x3x3 convolution of the warm-start network on the fifth-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory), sm_103a.
//
// Implicit GEMM: M = output voxels, N = output channels, K = 27 taps x input
// channels.  A block computes one tile of 128 output voxels (16 rows of 8
// voxels of one z plane of one cell) for all output channels.  Instead of
// gathering an im2col matrix per tap, it stages the tile's halo once in
// shared memory: 3 planes x 18 rows x 10 voxels of 16-byte channel chunks,
// laid out so that every tap's A operand is the same canonical no-swizzle
// K-major layout (8-row core matrices of 16-byte rows) at a different start
// address: rows of 8 voxels are 16 bytes apart, the 16 rows of the tile 160
// bytes apart (SBO) and consecutive 8-channel chunks 8640 bytes apart (LBO).
// The 27 taps then cost 27 x K/16 MMA instructions and no extra copies.
// The B operand (the tap's weights, K-major [cout][cin]) streams through two
// shared-memory stages; tcgen05.commit on a per-stage mbarrier tells the
// block when the MMAs that read a stage are done.  One thread issues the
// MMAs; the accumulator (128 lanes x N FP32 columns) stays in tensor memory
// until the epilogue reads it back with tcgen05.ld (warp w owns lanes
// 32w .. 32w + 31), adds the bias, applies the leaky ReLU and stores.
// Padding as the rest of the network: periodic in x and y, zero in z.
//
// Every wait on an mbarrier is bounded: on expiry the kernel records an
// error word (read by lbm_nn_tc_error), waits (bounded again) for the MMAs
// it issued, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int TILE_Y = 16, TILE_X = 8;             // 128 output voxels per block
constexpr int HZ = 3, HY = TILE_Y + 2, HX = TILE_X + 2;
constexpr int HALO_VOX = HZ * HY * HX;             // 540
constexpr int THREADS = 128;
constexpr int NSTAGE = 2;                          // weight stages
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

// Shared memory: halo [cg/8][3][18][10] x 16 B, then NSTAGE weight stages
// [cg/8][N/8][8] x 16 B, then the mbarriers and the TMEM address.
__host__ __device__ constexpr size_t tc_smem_bytes(int cg, int n) {
    return (size_t)HALO_VOX * cg * 2 + (size_t)NSTAGE * n * cg * 2 + 64;
}

// The bytes the kernel's descriptors can reach, whichever way the hardware
// reads the two strides: the layout needs tc_smem_bytes; the launch rounds
// the allocation up so that even the A operand walked with its strides
// exchanged (15 x 8640 bytes across the tile's rows) stays inside it.
__host__ __device__ constexpr size_t tc_smem_padded(int cg, int n) {
    return tc_smem_bytes(cg, n) + (size_t)15 * HALO_VOX * 16;
}

template <bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(THREADS) conv3_tc_kernel(const bf16* __restrict__ X, int Cin, int CG,
                                                           const bf16* __restrict__ Wk,
                                                           const float* __restrict__ bias,
                                                           void* __restrict__ Yv, int N, int tmem_cols,
                                                           Vol vol) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int CG8 = CG >> 3;
    unsigned char* halo = smem;
    unsigned char* wst = smem + (size_t)HALO_VOX * CG * 2;
    const size_t wstage_bytes = (size_t)N * CG * 2;
    unsigned long long* bars = reinterpret_cast<unsigned long long*>(wst + NSTAGE * wstage_bytes);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bars + NSTAGE);
    const unsigned halo_s = smem_u32(halo), wst_s = smem_u32(wst);

    // tile coordinates
    const int tiles_x = vol.w / TILE_X, tiles_y = vol.h / TILE_Y;
    int b = blockIdx.x;
    const int tx = b % tiles_x; b /= tiles_x;
    const int ty = b % tiles_y; b /= tiles_y;
    const int z0 = b % vol.d;
    const int n0 = b / vol.d;
    const int x0 = tx * TILE_X, y0 = ty * TILE_Y;

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(smem_u32(&bars[s]), 1);
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
    const uint32_t idesc = instr_desc(N);
    const unsigned lbo_a = HALO_VOX * 16, sbo_a = HX * 16;
    const unsigned lbo_b = (unsigned)(N / 8) * 128, sbo_b = 128;

    // Waits on the mbarriers are done by thread 0 alone (bounded); it
    // publishes a timeout through s_fail, which every thread reads after the
    // next __syncthreads, so all threads leave the loops together.
    __shared__ int s_fail;
    if (tid == 0) s_fail = 0;
    int issued = 0;                                 // MMA batches committed (one per tap)
    const int ngroups = Cin / CG;
    auto wait_batch = [&](int T) {                  // thread 0: batch T's MMAs are done
        if (tid == 0 && !s_fail &&
            !mbar_wait(smem_u32(&bars[T % NSTAGE]), (unsigned)((T / NSTAGE) & 1)))
            s_fail = 1;
    };
    auto load_weights = [&](int g, int t, int stage) {
        const bf16* wsrc = Wk + (long long)t * N * Cin + g * CG;
        const unsigned dst0 = wst_s + stage * (unsigned)wstage_bytes;
        for (int i = tid; i < N * CG8; i += THREADS) {
            const int co = i / CG8, c8 = i - co * CG8;
            cp16(dst0 + (unsigned)(((c8 * (N / 8) + (co >> 3)) * 8 + (co & 7)) * 16),
                 wsrc + (long long)co * Cin + c8 * 8, 16u);
        }
    };
    for (int g = 0; g < ngroups; ++g) {
        // the MMAs of the previous group read the halo and both stages
        if (g > 0) wait_batch(issued - 1);
        __syncthreads();
        if (s_fail) break;
        // halo of this channel group, and the weights of its first tap
        for (int i = tid; i < HALO_VOX * CG8; i += THREADS) {
            const int hv = i / CG8, c8 = i - hv * CG8;
            const int xh = hv % HX, yh = (hv / HX) % HY, zz = hv / (HX * HY);
            const int z = z0 + zz - 1;
            int y = y0 + yh - 1, x = x0 + xh - 1;
            y = y < 0 ? y + vol.h : (y >= vol.h ? y - vol.h : y);
            x = x < 0 ? x + vol.w : (x >= vol.w ? x - vol.w : x);
            const bool in = z >= 0 && z < vol.d;
            const long long v = (((long long)n0 * vol.d + (in ? z : 0)) * vol.h + y) * vol.w + x;
            cp16(halo_s + (unsigned)((((c8 * HZ + zz) * HY + yh) * HX + xh) * 16),
                 X + v * Cin + g * CG + c8 * 8, in ? 16u : 0u);
        }
        load_weights(g, 0, issued % NSTAGE);
        cp_commit();
        for (int t = 0; t < 27; ++t) {
            const int stage = issued % NSTAGE;
            cp_wait_all();                          // this thread's copies of tap t (and halo)
            fence_proxy_async();                    // visible to the tensor core's async proxy
            __syncthreads();
            if (s_fail) break;
            if (tid == 0) {
                fence_after();
                const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;
                const unsigned a0 = halo_s + (unsigned)(((dz * HY + dy) * HX + dx) * 16);
                const unsigned b0 = wst_s + stage * (unsigned)wstage_bytes;
                for (int ks = 0; ks < CG / 16; ++ks) {
                    const uint64_t ad = smem_desc(a0 + 2u * ks * lbo_a, lbo_a, sbo_a);
                    const uint64_t bd = smem_desc(b0 + 2u * ks * lbo_b, lbo_b, sbo_b);
                    mma_bf16(tmem, ad, bd, idesc, (g > 0 || t > 0 || ks > 0) ? 1u : 0u);
                }
                mma_commit(smem_u32(&bars[stage]));
            }
            ++issued;
            // the next tap's weights go to the other stage once the MMAs that
            // last read it (batch issued - NSTAGE) are done
            if (t + 1 < 27) {
                if (issued >= NSTAGE) wait_batch(issued - NSTAGE);
                __syncthreads();
                if (s_fail) break;
                load_weights(g, t + 1, issued % NSTAGE);
                cp_commit();
            }
        }
        if (s_fail) break;
    }
    cp_wait_all();
    // every MMA is done once the last batch's barrier completes (a second
    // bounded wait after a timeout, before the tensor memory is freed)
    if (issued > 0 && tid == 0) {
        const int T = issued - 1;
        if (!mbar_wait(smem_u32(&bars[T % NSTAGE]), (unsigned)((T / NSTAGE) & 1))) s_fail = 1;
    }
    __syncthreads();
    const bool failed = s_fail != 0;
    fence_after();
    if (failed) {
        atomicCAS(&g_tc_error, 0u, 1u);
    } else {
        // epilogue: lane m of the accumulator is output voxel m of the tile
        const int m = warp * 32 + lane;
        const int yy = m / TILE_X, xx = m % TILE_X;
        const long long v = (((long long)n0 * vol.d + z0) * vol.h + y0 + yy) * vol.w + x0 + xx;
        const unsigned trow = tmem + ((unsigned)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
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
                for (int q = 0; q < 4; ++q)
                    dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            } else {
                __align__(16) __nv_bfloat162 o[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) o[q] = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
                uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(Yv) + v * N + c0);
                dst[0] = *reinterpret_cast<const uint4*>(&o[0]);
                dst[1] = *reinterpret_cast<const uint4*>(&o[4]);
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols)
                     : "memory");
}

// Wk[tap][co][ci] = W[tap][ci][co] (forward), or W[26 - tap][co][ci] with
// the roles of ci and co swapped (the data gradient's conv: input channels
// co, output channels ci): Wk[tap][ci][co] = W[26 - tap][ci][co].
__global__ void kmajor_kernel(const bf16* __restrict__ W, bf16* __restrict__ Wk, int Cin, int Cout,
                              int flip) {
    const long long total = 27LL * Cin * Cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        if (!flip) {
            const int ci = (int)(i % Cin);
            const long long r = i / Cin;
            const int co = (int)(r % Cout);
            const int tap = (int)(r / Cout);
            Wk[i] = W[((long long)tap * Cin + ci) * Cout + co];
        } else {
            const int co = (int)(i % Cout);
            const long long r = i / Cout;
            const int ci = (int)(r % Cin);
            const int tap = (int)(r / Cin);
            Wk[i] = W[((long long)(26 - tap) * Cin + ci) * Cout + co];
        }
    }
}

int tmem_cols_for(int n) {
    int c = 32;
    while (c < n) c <<= 1;
    return c;
}

}  // namespace

extern "C" {

int lbm_nn_conv3d_tc_supported(int cin, int cout, int n, int d, int h, int w) {
    if (cin < 16 || cin % 16 || cout < 16 || cout % 16 || cout > 256) return 0;
    if (n < 1 || d < 1 || h < TILE_Y || w < TILE_X || h % TILE_Y || w % TILE_X) return 0;
    if ((long long)n * d * h * w >= (1LL << 40)) return 0;
    const int cg = cin <= 64 ? cin : (cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16));
    return tc_smem_padded(cg, cout) + 256 <= 227 * 1024 ? 1 : 0;   // static shared memory too
}

lbm_status lbm_nn_conv3d_tc(const void* x, int cin, const void* wk, const float* bias, void* y, int cout,
                            int n, int d, int h, int wdt, int relu, int out_f32, void* stream) {
    if (!x || !wk || !y || !lbm_nn_conv3d_tc_supported(cin, cout, n, d, h, wdt)) return LBM_ERR_INVALID_ARG;
    const int cg = cin <= 64 ? cin : (cin % 64 == 0 ? 64 : (cin % 32 == 0 ? 32 : 16));
    const size_t smem = tc_smem_padded(cg, cout);
    const Vol vol{n, d, h, wdt};
    const long long blocks = (long long)(wdt / TILE_X) * (h / TILE_Y) * d * n;
    if (blocks > 0x7fffffffLL) return LBM_ERR_INVALID_ARG;
    const int cols = tmem_cols_for(cout);
    cudaStream_t st = (cudaStream_t)stream;
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* W = static_cast<const bf16*>(wk);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) kern<<<(unsigned)blocks, THREADS, smem, st>>>(X, cin, cg, W, bias, y, cout, cols, vol);
    };
    if (relu && !out_f32) go(conv3_tc_kernel<true, false>);
    else if (!relu && !out_f32) go(conv3_tc_kernel<false, false>);
    else if (relu) go(conv3_tc_kernel<true, true>);
    else go(conv3_tc_kernel<false, true>);
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
