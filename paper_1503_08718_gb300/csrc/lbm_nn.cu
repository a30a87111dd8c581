// Layers of the learned warm-start network on the tensor cores.
//
// The network (a small 3D encoder-decoder, specified in the header) predicts
// the steady temperature of a cell from its material field; the lattice
// Boltzmann iteration then starts from f^eq of that prediction instead of the
// linear profile and still decides the answer (the paper's method only
// needs a steady state, Section 2.3).  Every layer here works on channels-last
// BF16 activations [voxel][channel] with FP32 accumulation:
//
//   conv: 3x3x3 (or 1x1x1) cross-correlation as an implicit GEMM
//         M = voxels, N = output channels, K = taps x input channels, on the
//         tensor cores with mma.sync m16n8k16 (BF16 in, FP32 accumulate);
//         periodic padding in x and y, zero padding in z; bias and leaky ReLU
//         (slope 0.01 below zero) fused
//   wgrad: dW[tap][ci][co] = sum_v X[v + tap][ci] dY[v][co], the same tensor
//         core tiles with the voxel axis as the reduction
//   data gradient: the forward conv with flipped taps and swapped channels
//   pooling, nearest upsampling, concatenation, the 1x1x1 head fused with the
//   squared-error loss, and Adam on FP32 master weights.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "lbm.h"

namespace {

using bf16 = __nv_bfloat16;

struct Vol {
    int n, d, h, w;
};

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                       unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                         unsigned& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma16816(float (&d)[4], unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Source voxel of tap (dz, dy, dx) in {0,1,2}^3 for voxel (n, z, y, x):
// periodic in x and y, -1 (zero) outside in z.
__device__ __forceinline__ long long tap_src(const Vol& v, int n, int z, int y, int x, int dz, int dy,
                                             int dx) {
    const int zs = z + dz - 1;
    if (zs < 0 || zs >= v.d) return -1;
    int ys = y + dy - 1, xs = x + dx - 1;
    ys = ys < 0 ? ys + v.h : (ys >= v.h ? ys - v.h : ys);
    xs = xs < 0 ? xs + v.w : (xs >= v.w ? xs - v.w : xs);
    return (((long long)n * v.d + zs) * v.h + ys) * v.w + xs;
}

constexpr int BM = 128;     // voxels per block (4 warps x 32)
// leaky ReLU slope for negative inputs (a plain ReLU can die under Adam)
constexpr float kLeak = 0.01f;
constexpr int NT = 128;     // threads

// Y[v][co] = act(bias[co] + sum_tap sum_ci X[src(v, tap)][ci] W[tap][ci][co])
template <int BN, int BK, int KS, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(NT) conv_fwd_kernel(const bf16* __restrict__ X, int Cin,
                                                      const bf16* __restrict__ W,
                                                      const float* __restrict__ bias,
                                                      void* __restrict__ Yv, int Cout, Vol vol) {
    __shared__ __align__(16) bf16 sA[BM][BK + 8];
    __shared__ __align__(16) bf16 sB[BK][BN + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long V = (long long)vol.n * vol.d * vol.h * vol.w;
    const long long v0 = (long long)blockIdx.x * BM;
    const int n0 = blockIdx.y * BN;
    // this thread stages row `tid` of the A tile
    const long long vr = v0 + tid;
    int rn = 0, rz = 0, ry = 0, rx = 0;
    if (vr < V) {
        long long t = vr;
        rx = (int)(t % vol.w); t /= vol.w;
        ry = (int)(t % vol.h); t /= vol.h;
        rz = (int)(t % vol.d); rn = (int)(t / vol.d);
    }
    float acc[2][BN / 8][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < BN / 8; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    constexpr int TAPS = KS * KS * KS;
    for (int tap = 0; tap < TAPS; ++tap) {
        const int dz = KS == 3 ? tap / 9 : 1, dy = KS == 3 ? (tap / 3) % 3 : 1, dx = KS == 3 ? tap % 3 : 1;
        const long long src = vr < V ? tap_src(vol, rn, rz, ry, rx, dz, dy, dx) : -1;
        for (int c0 = 0; c0 < Cin; c0 += BK) {
            // A: one voxel row of BK channels per thread
#pragma unroll
            for (int q = 0; q < BK / 8; ++q) {
                uint4 val = make_uint4(0u, 0u, 0u, 0u);
                if (src >= 0) val = *reinterpret_cast<const uint4*>(X + src * Cin + c0 + 8 * q);
                *reinterpret_cast<uint4*>(&sA[tid][8 * q]) = val;
            }
            // B: BK rows of BN output channels
            for (int i = tid; i < BK * (BN / 8); i += NT) {
                const int r = i / (BN / 8), q = i % (BN / 8);
                const bf16* wp = W + ((long long)tap * Cin + c0 + r) * Cout + n0 + 8 * q;
                *reinterpret_cast<uint4*>(&sB[r][8 * q]) = *reinterpret_cast<const uint4*>(wp);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; kk += 16) {
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
                    ldm_x4(smem_addr(&sA[warp * 32 + mt * 16 + (lane & 15)][kk + (lane >> 4) * 8]),
                           a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
#pragma unroll
                for (int nt = 0; nt < BN / 8; nt += 2) {
                    const int mi = lane >> 3;
                    unsigned b0, b1, b2, b3;
                    ldm_x4_t(smem_addr(&sB[kk + (mi & 1) * 8 + (lane & 7)][nt * 8 + (mi >> 1) * 8]),
                             b0, b1, b2, b3);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma16816(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                        mma16816(acc[mt][nt + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                    }
                }
            }
            __syncthreads();
        }
    }
    // epilogue: bias, activation, store
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < BN / 8; ++nt)
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const long long v = v0 + warp * 32 + mt * 16 + (lane >> 2) + 8 * half;
                if (v >= V) continue;
                const int co = n0 + nt * 8 + (lane & 3) * 2;
                float y0 = acc[mt][nt][2 * half] + (bias ? bias[co] : 0.f);
                float y1 = acc[mt][nt][2 * half + 1] + (bias ? bias[co + 1] : 0.f);
                if (RELU) {
                    y0 = y0 > 0.f ? y0 : kLeak * y0;
                    y1 = y1 > 0.f ? y1 : kLeak * y1;
                }
                if (OUT_F32) {
                    float* Y = reinterpret_cast<float*>(Yv);
                    *reinterpret_cast<float2*>(Y + v * Cout + co) = make_float2(y0, y1);
                } else {
                    bf16* Y = reinterpret_cast<bf16*>(Yv);
                    *reinterpret_cast<__nv_bfloat162*>(Y + v * Cout + co) = __floats2bfloat162_rn(y0, y1);
                }
            }
}

// dW[tap][ci][co] += sum over a chunk of voxels of X[src(v, tap)][ci] G[v][co]
// (M = 64 input channels, N = BN output channels, K = voxels in steps of 32).
constexpr int WG_CHUNK = 4096;   // voxels per block
template <int BN, int KS>
__global__ void __launch_bounds__(NT) conv_wgrad_kernel(const bf16* __restrict__ X, int Cin,
                                                        const bf16* __restrict__ G, int Cout,
                                                        float* __restrict__ dW, Vol vol) {
    constexpr int BMc = 64, BKv = 32;
    __shared__ __align__(16) bf16 sX[BKv][BMc + 8];
    __shared__ __align__(16) bf16 sG[BKv][BN + 8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long V = (long long)vol.n * vol.d * vol.h * vol.w;
    const int nco = Cout / BN;
    const int tap = blockIdx.z / nco;
    const int n0 = (blockIdx.z % nco) * BN;
    const int ci0 = blockIdx.y * BMc;
    const int cw = Cin - ci0 < BMc ? Cin - ci0 : BMc;    // 16, 32 or 64 live channels
    const long long vbeg = (long long)blockIdx.x * WG_CHUNK;
    const long long vend = vbeg + WG_CHUNK < V ? vbeg + WG_CHUNK : V;
    const int dz = KS == 3 ? tap / 9 : 1, dy = KS == 3 ? (tap / 3) % 3 : 1, dx = KS == 3 ? tap % 3 : 1;
    float acc[BN / 8][4];
#pragma unroll
    for (int j = 0; j < BN / 8; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[j][k] = 0.f;
    for (long long vb = vbeg; vb < vend; vb += BKv) {
        // X rows (shifted by the tap) and G rows for BKv voxels
        for (int i = tid; i < BKv * (BMc / 8); i += NT) {
            const int r = i / (BMc / 8), q = i % (BMc / 8);
            const long long v = vb + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < vend && 8 * q < cw) {
                long long t = v;
                const int x = (int)(t % vol.w); t /= vol.w;
                const int y = (int)(t % vol.h); t /= vol.h;
                const int z = (int)(t % vol.d); const int n = (int)(t / vol.d);
                const long long s = tap_src(vol, n, z, y, x, dz, dy, dx);
                if (s >= 0) val = *reinterpret_cast<const uint4*>(X + s * Cin + ci0 + 8 * q);
            }
            *reinterpret_cast<uint4*>(&sX[r][8 * q]) = val;
        }
        for (int i = tid; i < BKv * (BN / 8); i += NT) {
            const int r = i / (BN / 8), q = i % (BN / 8);
            const long long v = vb + r;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < vend) val = *reinterpret_cast<const uint4*>(G + v * Cout + n0 + 8 * q);
            *reinterpret_cast<uint4*>(&sG[r][8 * q]) = val;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BKv; kk += 16) {
            // A = X^T: rows are channels (warp's 16), columns voxels
            const int mi = lane >> 3;
            unsigned a0, a1, a2, a3;
            ldm_x4_t(smem_addr(&sX[kk + (mi >> 1) * 8 + (lane & 7)][warp * 16 + (mi & 1) * 8]), a0, a1,
                     a2, a3);
#pragma unroll
            for (int nt = 0; nt < BN / 8; nt += 2) {
                unsigned b0, b1, b2, b3;
                ldm_x4_t(smem_addr(&sG[kk + (mi & 1) * 8 + (lane & 7)][nt * 8 + (mi >> 1) * 8]), b0, b1,
                         b2, b3);
                mma16816(acc[nt], a0, a1, a2, a3, b0, b1);
                mma16816(acc[nt + 1], a0, a1, a2, a3, b2, b3);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int nt = 0; nt < BN / 8; ++nt)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int ci = ci0 + warp * 16 + (lane >> 2) + 8 * half;
            if (ci >= ci0 + cw) continue;
            const int co = n0 + nt * 8 + (lane & 3) * 2;
            float* p = dW + ((long long)tap * Cin + ci) * Cout + co;
            atomicAdd(p, acc[nt][2 * half]);
            atomicAdd(p + 1, acc[nt][2 * half + 1]);
        }
}

// Wf[tap][co][ci] = W[taps-1-tap][ci][co] (the data gradient's weights).
__global__ void flip_kernel(const bf16* __restrict__ W, bf16* __restrict__ Wf, int Cin, int Cout,
                            int taps) {
    const long long total = (long long)taps * Cin * Cout;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ci = (int)(i % Cin);
        const long long r = i / Cin;
        const int co = (int)(r % Cout);
        const int tap = (int)(r / Cout);
        Wf[i] = W[((long long)(taps - 1 - tap) * Cin + ci) * Cout + co];
    }
}

__global__ void bias_grad_kernel(const bf16* __restrict__ G, int C, long long V,
                                 float* __restrict__ db) {
    // blockDim.x >= C; each block sums a chunk of voxels per channel
    const int c = threadIdx.x;
    if (c >= C) return;
    float s = 0.f;
    const long long chunk = (V + gridDim.x - 1) / gridDim.x;
    const long long vb = blockIdx.x * chunk;
    const long long ve = vb + chunk < V ? vb + chunk : V;
    for (long long v = vb; v < ve; ++v) s += __bfloat162float(G[v * C + c]);
    atomicAdd(db + c, s);
}

__global__ void relu_mask_kernel(const bf16* __restrict__ dY, const bf16* __restrict__ Y,
                                 bf16* __restrict__ G, long long count) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        G[i] = __bfloat162float(Y[i]) > 0.f ? dY[i] : __float2bfloat16(kLeak * __bfloat162float(dY[i]));
}

// out[parent][c] = scale * sum of the 8 children (input dims are the children's)
__global__ void pool2_kernel(const bf16* __restrict__ X, bf16* __restrict__ Y, int C, Vol vin,
                             float scale) {
    const int d2 = vin.d / 2, h2 = vin.h / 2, w2 = vin.w / 2;
    const long long total = (long long)vin.n * d2 * h2 * w2 * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long t = i / C;
        const int x = (int)(t % w2); t /= w2;
        const int y = (int)(t % h2); t /= h2;
        const int z = (int)(t % d2); const int n = (int)(t / d2);
        float s = 0.f;
        for (int k = 0; k < 8; ++k) {
            const long long src = (((long long)n * vin.d + 2 * z + (k >> 2)) * vin.h + 2 * y + ((k >> 1) & 1)) *
                                      vin.w + 2 * x + (k & 1);
            s += __bfloat162float(X[src * C + c]);
        }
        Y[i] = __float2bfloat16(scale * s);
    }
}

// out[child][c] = scale * in[parent][c] (output dims are the children's)
__global__ void upsample2_kernel(const bf16* __restrict__ X, bf16* __restrict__ Y, int C, Vol vout,
                                 float scale) {
    const long long total = (long long)vout.n * vout.d * vout.h * vout.w * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        long long t = i / C;
        const int x = (int)(t % vout.w); t /= vout.w;
        const int y = (int)(t % vout.h); t /= vout.h;
        const int z = (int)(t % vout.d); const int n = (int)(t / vout.d);
        const long long src = (((long long)n * (vout.d / 2) + z / 2) * (vout.h / 2) + y / 2) * (vout.w / 2) + x / 2;
        Y[i] = __float2bfloat16(scale * __bfloat162float(X[src * C + c]));
    }
}

__global__ void concat_kernel(const bf16* __restrict__ A, int ca, const bf16* __restrict__ B, int cb,
                              bf16* __restrict__ Y, long long V) {
    const int C = ca + cb;
    const long long total = V * C;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        const long long v = i / C;
        Y[i] = c < ca ? A[v * ca + c] : B[v * cb + c - ca];
    }
}

// dst[v][c] (+)= src[v][off + c]
__global__ void slice_kernel(const bf16* __restrict__ S, int cs, int off, bf16* __restrict__ D, int c,
                             long long V, int accumulate) {
    const long long total = V * c;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % c);
        const long long v = i / c;
        float s = __bfloat162float(S[v * cs + off + k]);
        if (accumulate) s += __bfloat162float(D[i]);
        D[i] = __float2bfloat16(s);
    }
}

// 1x1x1 head to one channel with the squared-error loss:
// T = T_lin + b + w . h;  loss += (T - target)^2;  dT = 2 (T - target) / count;
// dh = dT w (bf16);  dw += dT h;  db += dT.  Without a target only T is written.
constexpr int HEAD_C = 32;
__global__ void head_kernel(const bf16* __restrict__ H, const float* __restrict__ w,
                            const float* __restrict__ b, const float* __restrict__ t_lin,
                            const float* __restrict__ target, float* __restrict__ pred,
                            bf16* __restrict__ dH, float* __restrict__ dw, float* __restrict__ db,
                            double* __restrict__ loss, long long V, double inv_count) {
    __shared__ float s_w[HEAD_C];
    __shared__ float s_dw[HEAD_C + 1];
    __shared__ double s_loss;
    if (threadIdx.x < HEAD_C) s_w[threadIdx.x] = w[threadIdx.x];
    if (threadIdx.x <= HEAD_C) s_dw[threadIdx.x] = 0.f;
    if (threadIdx.x == 0) s_loss = 0.0;
    __syncthreads();
    float ldw[HEAD_C];
#pragma unroll
    for (int c = 0; c < HEAD_C; ++c) ldw[c] = 0.f;
    float ldb = 0.f;
    double lloss = 0.0;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        float h[HEAD_C];
        const uint4* hp = reinterpret_cast<const uint4*>(H + v * HEAD_C);
#pragma unroll
        for (int q = 0; q < HEAD_C / 8; ++q) {
            const uint4 u = hp[q];
            const __nv_bfloat162* p2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(p2[e]);
                h[8 * q + 2 * e] = f.x;
                h[8 * q + 2 * e + 1] = f.y;
            }
        }
        float T = t_lin[v] + b[0];
#pragma unroll
        for (int c = 0; c < HEAD_C; ++c) T = fmaf(s_w[c], h[c], T);
        pred[v] = T;
        if (target) {
            const float diff = T - target[v];
            lloss += (double)diff * (double)diff;
            const float g = (float)(2.0 * inv_count) * diff;
            ldb += g;
            uint4 out[HEAD_C / 8];
#pragma unroll
            for (int q = 0; q < HEAD_C / 8; ++q) {
                __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(&out[q]);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    o2[e] = __floats2bfloat162_rn(g * s_w[8 * q + 2 * e], g * s_w[8 * q + 2 * e + 1]);
            }
            uint4* dp = reinterpret_cast<uint4*>(dH + v * HEAD_C);
#pragma unroll
            for (int q = 0; q < HEAD_C / 8; ++q) dp[q] = out[q];
#pragma unroll
            for (int c = 0; c < HEAD_C; ++c) ldw[c] = fmaf(g, h[c], ldw[c]);
        }
    }
    if (!target) return;
#pragma unroll
    for (int c = 0; c < HEAD_C; ++c) atomicAdd(&s_dw[c], ldw[c]);
    atomicAdd(&s_dw[HEAD_C], ldb);
    atomicAdd(&s_loss, lloss);
    __syncthreads();
    if (threadIdx.x < HEAD_C) atomicAdd(dw + threadIdx.x, s_dw[threadIdx.x]);
    if (threadIdx.x == HEAD_C) atomicAdd(db, s_dw[HEAD_C]);
    if (threadIdx.x == 0) atomicAdd(loss, s_loss);
}

// Network input: 6 tensor components of the voxel's phase (normalised) and
// the linear profile of its plane; channels 7..15 are zero.
__global__ void input_kernel(const uint8_t* __restrict__ phase, const float* __restrict__ table,
                             const float* __restrict__ t_lin_z, bf16* __restrict__ X, Vol vol) {
    const long long V = (long long)vol.n * vol.d * vol.h * vol.w;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        const int z = (int)((v / ((long long)vol.w * vol.h)) % vol.d);
        const float* t = table + 6 * phase[v];
        __align__(16) bf16 ch[16];
#pragma unroll
        for (int c = 0; c < 6; ++c) ch[c] = __float2bfloat16(t[c]);
        ch[6] = __float2bfloat16(t_lin_z[z]);
#pragma unroll
        for (int c = 7; c < 16; ++c) ch[c] = __float2bfloat16(0.f);
        uint4* dst = reinterpret_cast<uint4*>(X + v * 16);
        dst[0] = *reinterpret_cast<const uint4*>(&ch[0]);
        dst[1] = *reinterpret_cast<const uint4*>(&ch[8]);
    }
}

// Adam on FP32 master weights; writes the BF16 copy the layers read.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, bf16* __restrict__ pb, long long count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16(pi);
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    if (g > 152LL * 16) g = 152LL * 16;
    return (int)(g < 1 ? 1 : g);
}

template <int BN, int BK, int KS>
void conv_dispatch(const bf16* X, int Cin, const bf16* W, const float* b, void* Y, int Cout, Vol vol,
                   bool relu, bool out_f32, cudaStream_t st) {
    const long long V = (long long)vol.n * vol.d * vol.h * vol.w;
    const dim3 grid((unsigned)((V + BM - 1) / BM), (unsigned)(Cout / BN));
    if (relu && !out_f32) conv_fwd_kernel<BN, BK, KS, true, false><<<grid, NT, 0, st>>>(X, Cin, W, b, Y, Cout, vol);
    else if (!relu && !out_f32) conv_fwd_kernel<BN, BK, KS, false, false><<<grid, NT, 0, st>>>(X, Cin, W, b, Y, Cout, vol);
    else if (relu) conv_fwd_kernel<BN, BK, KS, true, true><<<grid, NT, 0, st>>>(X, Cin, W, b, Y, Cout, vol);
    else conv_fwd_kernel<BN, BK, KS, false, true><<<grid, NT, 0, st>>>(X, Cin, W, b, Y, Cout, vol);
}

lbm_status status_of(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ERR_CUDA; }

bool vol_ok(int n, int d, int h, int w) {
    return n >= 1 && d >= 1 && h >= 1 && w >= 1 && (long long)n * d * h * w < (1LL << 40);
}

}  // namespace

extern "C" {

lbm_status lbm_nn_conv3d(const void* x, int cin, const void* w, const float* bias, void* y, int cout,
                         int n, int d, int h, int wdt, int ksize, int relu, int out_f32,
                         void* stream) {
    if (!x || !w || !y || cin < 16 || cin % 16 || cout < 32 || cout % 32 || !vol_ok(n, d, h, wdt) ||
        (ksize != 1 && ksize != 3))
        return LBM_ERR_INVALID_ARG;
    const Vol vol{n, d, h, wdt};
    cudaStream_t st = (cudaStream_t)stream;
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* W = static_cast<const bf16*>(w);
    const bool r = relu != 0, o = out_f32 != 0;
    const bool bk32 = cin % 32 == 0, bn64 = cout % 64 == 0;
    if (ksize == 3) {
        if (bn64 && bk32) conv_dispatch<64, 32, 3>(X, cin, W, bias, y, cout, vol, r, o, st);
        else if (bn64) conv_dispatch<64, 16, 3>(X, cin, W, bias, y, cout, vol, r, o, st);
        else if (bk32) conv_dispatch<32, 32, 3>(X, cin, W, bias, y, cout, vol, r, o, st);
        else conv_dispatch<32, 16, 3>(X, cin, W, bias, y, cout, vol, r, o, st);
    } else {
        if (bn64 && bk32) conv_dispatch<64, 32, 1>(X, cin, W, bias, y, cout, vol, r, o, st);
        else if (bn64) conv_dispatch<64, 16, 1>(X, cin, W, bias, y, cout, vol, r, o, st);
        else if (bk32) conv_dispatch<32, 32, 1>(X, cin, W, bias, y, cout, vol, r, o, st);
        else conv_dispatch<32, 16, 1>(X, cin, W, bias, y, cout, vol, r, o, st);
    }
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_conv3d_wgrad(const void* x, int cin, const void* g, int cout, float* dw, int n,
                               int d, int h, int wdt, int ksize, void* stream) {
    if (!x || !g || !dw || cin < 16 || cin % 16 || cout < 32 || cout % 32 || !vol_ok(n, d, h, wdt) ||
        (ksize != 1 && ksize != 3))
        return LBM_ERR_INVALID_ARG;
    const Vol vol{n, d, h, wdt};
    const long long V = (long long)n * d * h * wdt;
    const int taps = ksize * ksize * ksize;
    cudaStream_t st = (cudaStream_t)stream;
    const bf16* X = static_cast<const bf16*>(x);
    const bf16* G = static_cast<const bf16*>(g);
    const unsigned chunks = (unsigned)((V + WG_CHUNK - 1) / WG_CHUNK);
    const unsigned cib = (unsigned)((cin + 63) / 64);
    if (cout % 64 == 0) {
        const dim3 grid(chunks, cib, (unsigned)(taps * (cout / 64)));
        if (ksize == 3) conv_wgrad_kernel<64, 3><<<grid, NT, 0, st>>>(X, cin, G, cout, dw, vol);
        else conv_wgrad_kernel<64, 1><<<grid, NT, 0, st>>>(X, cin, G, cout, dw, vol);
    } else {
        const dim3 grid(chunks, cib, (unsigned)(taps * (cout / 32)));
        if (ksize == 3) conv_wgrad_kernel<32, 3><<<grid, NT, 0, st>>>(X, cin, G, cout, dw, vol);
        else conv_wgrad_kernel<32, 1><<<grid, NT, 0, st>>>(X, cin, G, cout, dw, vol);
    }
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_flip_weights(const void* w, void* wf, int cin, int cout, int ksize, void* stream) {
    if (!w || !wf || cin < 1 || cout < 1 || (ksize != 1 && ksize != 3)) return LBM_ERR_INVALID_ARG;
    const int taps = ksize * ksize * ksize;
    flip_kernel<<<grid_for((long long)taps * cin * cout), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(w), static_cast<bf16*>(wf), cin, cout, taps);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_bias_grad(const void* g, int c, long long nvox, float* db, void* stream) {
    if (!g || !db || c < 1 || c > 1024 || nvox < 1) return LBM_ERR_INVALID_ARG;
    long long blocks = (nvox + 1023) / 1024;
    if (blocks > 152 * 8) blocks = 152 * 8;
    const int threads = (c + 31) / 32 * 32;
    bias_grad_kernel<<<(int)blocks, threads, 0, (cudaStream_t)stream>>>(static_cast<const bf16*>(g), c,
                                                                        nvox, db);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_relu_mask(const void* dy, const void* y, void* g, long long count, void* stream) {
    if (!dy || !y || !g || count < 0) return LBM_ERR_INVALID_ARG;
    relu_mask_kernel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(dy), static_cast<const bf16*>(y), static_cast<bf16*>(g), count);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_pool2(const void* x, void* y, int c, int n, int d, int h, int w, float scale,
                        void* stream) {
    if (!x || !y || c < 1 || !vol_ok(n, d, h, w) || (d | h | w) & 1) return LBM_ERR_INVALID_ARG;
    const Vol v{n, d, h, w};
    pool2_kernel<<<grid_for((long long)n * d * h * w * c / 8), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(x), static_cast<bf16*>(y), c, v, scale);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_upsample2(const void* x, void* y, int c, int n, int d, int h, int w, float scale,
                            void* stream) {
    if (!x || !y || c < 1 || !vol_ok(n, d, h, w) || (d | h | w) & 1) return LBM_ERR_INVALID_ARG;
    const Vol v{n, d, h, w};
    upsample2_kernel<<<grid_for((long long)n * d * h * w * c), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(x), static_cast<bf16*>(y), c, v, scale);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_concat(const void* a, int ca, const void* b, int cb, void* y, long long nvox,
                         void* stream) {
    if (!a || !b || !y || ca < 1 || cb < 1 || nvox < 1) return LBM_ERR_INVALID_ARG;
    concat_kernel<<<grid_for(nvox * (ca + cb)), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(a), ca, static_cast<const bf16*>(b), cb, static_cast<bf16*>(y), nvox);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_slice(const void* src, int csrc, int coff, void* dst, int c, long long nvox,
                        int accumulate, void* stream) {
    if (!src || !dst || c < 1 || coff < 0 || coff + c > csrc || nvox < 1) return LBM_ERR_INVALID_ARG;
    slice_kernel<<<grid_for(nvox * c), 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(src), csrc, coff, static_cast<bf16*>(dst), c, nvox, accumulate);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_head(const void* hdn, const float* w, const float* b, const float* t_lin,
                       const float* target, float* pred, void* dh, float* dw, float* db,
                       double* loss, long long nvox, void* stream) {
    if (!hdn || !w || !b || !t_lin || !pred || nvox < 1 ||
        (target && (!dh || !dw || !db || !loss)))
        return LBM_ERR_INVALID_ARG;
    long long blocks = (nvox + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    head_kernel<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(
        static_cast<const bf16*>(hdn), w, b, t_lin, target, pred, static_cast<bf16*>(dh), dw, db, loss,
        nvox, 1.0 / (double)nvox);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_input(const uint8_t* phase, const float* table, const float* t_lin_z, void* x,
                        int n, int d, int h, int w, void* stream) {
    if (!phase || !table || !t_lin_z || !x || !vol_ok(n, d, h, w)) return LBM_ERR_INVALID_ARG;
    const Vol v{n, d, h, w};
    input_kernel<<<grid_for((long long)n * d * h * w), 256, 0, (cudaStream_t)stream>>>(
        phase, table, t_lin_z, static_cast<bf16*>(x), v);
    return status_of(cudaGetLastError());
}

lbm_status lbm_nn_adam(float* p, const float* g, float* m, float* v, void* p_bf16, long long count,
                       float lr, float beta1, float beta2, float eps, int step, void* stream) {
    if (!p || !g || !m || !v || count < 1 || step < 1) return LBM_ERR_INVALID_ARG;
    const float c1 = 1.f / (1.f - powf(beta1, (float)step));
    const float c2 = 1.f / (1.f - powf(beta2, (float)step));
    adam_kernel<<<grid_for(count), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, static_cast<bf16*>(p_bf16),
                                                                   count, lr, beta1, beta2, eps, c1, c2);
    return status_of(cudaGetLastError());
}

}  // extern "C"
