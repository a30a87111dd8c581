// Device kernels of the D3Q7 MRT lattice Boltzmann hot path for sm_103a.
//
// Storage: structure of arrays f[i][z][y][x] (population-major), FP32, two
// buffers (pull scheme: read the previous post-collision state, write the
// next one).  The Dirichlet axis is always the slowest index z; the host lays
// the cell out that way.  Rows are padded to a multiple of 4 voxels (pitch)
// so that every thread moves one aligned 16-byte float4 per population.
// Values are stored as deviations g_i = f_i - w_i R(z), w_0 = 1/4,
// w_1..6 = 1/8 (Eq. 6 with gamma = 1/8), from a per-plane reference
// temperature R(z): the plane mean of T at the previous check, quantised to a
// power-of-two grid so that every frame-change constant w_i (R(z') - R(z)) is
// exact in FP32.  The map is linear, so the frame changes nothing in exact
// arithmetic; in FP32 the stored values are small (non-equilibrium parts and
// in-plane temperature variation), which shrinks the rounding of the stored
// state and with it the FP32 error of the converged fixed point.
//
// Collision (Eq. 5, 8-13).  With tau_0 = tau_4 = tau_5 = tau_6 = 1 the
// moments 0, 4, 5, 6 leave the collision at equilibrium and the flux moment
// j = (f1 - f2, f3 - f4, f5 - f6) relaxes to jhat = j - S_b j with
// S_b = tau^-1 (the 3x3 off-diagonal block of Eq. 12 inverted).  Because the
// rows of M in Eq. 11 are orthogonal, M^-1 maps this back to
//   fhat_0 = T / 4,   fhat_{2k-1,2k} = T / 8 +- jhat_k / 2,
// which is M^-1 S M applied exactly (no 7x7 product on the device).
// Interfaces need no code: each node uses its own phase's S_b and streaming
// is plain (Eq. 21, the half-lattice division scheme of Section 2.3).
//
// Flux (Eq. 15-16).  With D = eps (tau - I/2) and grad T = -tau^-1 j / eps,
// q = -D grad T = (I - S_b / 2) j = (j + jhat) / 2 at every node.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

constexpr int kThreads = 256;        // threads per step block
constexpr unsigned kFull = 0xffffffffu;

struct Ctl {
    long long iter;      // iterations since start
    long long iter_snap; // iteration of the temperature snapshot
    long long checks;
    double k_eff, r_t, r_q, best_rt;
    int status;          // lbm_status of the last check
    int since_best;
    int done;
    unsigned glob_cnt;   // planes closed in the current check (0 between checks)
};

// What the blocks that close a check need: per-plane and global reductions,
// the next reference frame and the stop rule.
struct CheckArgs {
    double* part;                    // block partials [4][nz][blocks_per_plane]
    double* Q;                       // plane flux sums [nz]
    double* plane;                   // per-plane sum |dT| [nz] and sum |T| [nz]
    int* plane_cnt;                  // closing tickets per plane [nz], 0 between checks
    Ctl* ctl;
    float* ra;                       // frame of the state between calls [nz]
    float* rb;                       // frame of the next interval [nz]
    float* rc;                       // staging of the new plane means [nz]
    int rebase;                      // the interval's first step moved the state to rb
    int steps;                       // iterations this check closes
    int stall_checks;
    int interval;                    // steps the next interval would add
    long long max_iters;
    double tol;
    double keff_scale;               // nz / (s * dT * nx * ny)
    double inv_area;                 // 1 / (nx * ny)
    double quantum, inv_quantum;     // grid of the reference values (power of two)
    cudaGraphConditionalHandle handle;
    int use_handle;
};

struct StepArgs {
    const float* __restrict__ src;   // 7 populations, post-collision state n-1
    float* __restrict__ dst;         // 7 populations, post-collision state n
    const uint8_t* __restrict__ phase;  // [nz][ny][pitch], padded with 0
    const float4* __restrict__ sb;   // 2 float4 per phase: (xx, yy, zz, yz), (xz, xy, -, -)
    float* __restrict__ tsnap;       // T - T_ref at the previous check, [nz][ny][pitch]
    const float* __restrict__ rsrc;  // reference R(z) of the src state, [nz]
    const float* __restrict__ rdst;  // reference R(z) of the dst state, [nz]
    long long pstride;               // floats per population = pitch * ny * nz
    int nx, ny, nz, pitch, n_phases;
    int quads_per_plane;             // (pitch / 4) * ny
    int blocks_per_plane;
    float eps_hot, eps_cold;         // eps * T_wall
    double t_ref;                    // offset of the residual snapshot
    CheckArgs ck;
};

__device__ __forceinline__ float4 ld4(const float* p) {
    return __ldg(reinterpret_cast<const float4*>(p));
}

__device__ __forceinline__ void st4(float* p, float4 v) {
    *reinterpret_cast<float4*>(p) = v;
}

__device__ __forceinline__ float comp(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

__device__ __forceinline__ void set_comp(float4& v, int k, float s) {
    if (k == 0) v.x = s;
    else if (k == 1) v.y = s;
    else if (k == 2) v.z = s;
    else v.w = s;
}

// Closing a check (Eq. 15-16 plane sums, Eq. 22, the stop rule).  Every
// block of a check step writes its FP64 partials and takes a ticket on its
// plane's counter; the block that takes the last ticket sums the plane's
// partials in block order, and the block that closes the last plane sums the
// planes in plane order and applies the stop rule.  No block ever waits:
// the work falls to whichever block finishes last, and the result is
// deterministic.

__device__ void close_check(const StepArgs& a) {
    const CheckArgs& ck = a.ck;
    double qsum = 0.0, qmax = -INFINITY, qmin = INFINITY, dsum = 0.0, tsum = 0.0;
    for (int z = threadIdx.x; z < a.nz; z += kThreads) {
        const double q = __ldcg(ck.Q + z);
        qsum += q;
        qmax = fmax(qmax, q);
        qmin = fmin(qmin, q);
        dsum += __ldcg(ck.plane + z);
        tsum += __ldcg(ck.plane + a.nz + z);
    }
    __shared__ double s[5][kThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        qsum += __shfl_down_sync(kFull, qsum, off);
        qmax = fmax(qmax, __shfl_down_sync(kFull, qmax, off));
        qmin = fmin(qmin, __shfl_down_sync(kFull, qmin, off));
        dsum += __shfl_down_sync(kFull, dsum, off);
        tsum += __shfl_down_sync(kFull, tsum, off);
    }
    if (lane == 0) {
        s[0][warp] = qsum; s[1][warp] = qmax; s[2][warp] = qmin; s[3][warp] = dsum; s[4][warp] = tsum;
    }
    __syncthreads();
    // rotate the reference frames: every block of this kernel has finished
    // reading them (their tickets were all taken)
    for (int z = threadIdx.x; z < a.nz; z += kThreads) {
        if (ck.rebase) ck.ra[z] = ck.rb[z];
        ck.rb[z] = __ldcg(ck.rc + z);
    }
    if (threadIdx.x == 0) {
        qsum = 0.0; qmax = -INFINITY; qmin = INFINITY; dsum = 0.0; tsum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) {
            qsum += s[0][w];
            qmax = fmax(qmax, s[1][w]);
            qmin = fmin(qmin, s[2][w]);
            dsum += s[3][w];
            tsum += s[4][w];
        }
        Ctl* c = ck.ctl;
        const double mean = qsum / (double)a.nz;
        c->iter += ck.steps;
        c->checks += 1;
        c->k_eff = ck.keff_scale * mean;
        c->r_q = (qmax - qmin) / fabs(mean);
        // mean per-step change of T since the previous check, relative to T
        c->r_t = dsum / ((double)(c->iter - c->iter_snap) * tsum);
        c->iter_snap = c->iter;
        int status;
        if (!isfinite(c->r_t) || !isfinite(c->k_eff)) {
            status = 6;                                   // LBM_ERR_DIVERGED
        } else if (c->r_t <= ck.tol) {
            status = 0;                                   // LBM_OK (converged)
        } else {
            if (c->r_t < c->best_rt) {
                c->best_rt = c->r_t;
                c->since_best = 0;
            } else {
                c->since_best += 1;
            }
            if (ck.stall_checks > 0 && c->since_best >= ck.stall_checks) status = 7;   // STALLED
            else status = 5;                              // LBM_ERR_NOT_CONVERGED (so far)
        }
        c->status = status;
        const bool stop = status != 5 || c->iter + ck.interval > ck.max_iters;
        c->done = stop ? 1 : 0;
        c->glob_cnt = 0u;
        if (ck.use_handle) cudaGraphSetConditional(ck.handle, stop ? 0u : 1u);
    }
}

__device__ void close_plane(const StepArgs& a, int z) {
    const CheckArgs& ck = a.ck;
    __shared__ int s_last_plane;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const long long plane_all = (long long)a.nz * a.blocks_per_plane;
        const long long base = (long long)z * a.blocks_per_plane;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = lane; b < a.blocks_per_plane; b += 32)
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] += __ldcg(ck.part + m * plane_all + base + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] += __shfl_down_sync(kFull, v[m], off);
        if (lane == 0) {
            ck.Q[z] = v[0];
            ck.plane[z] = v[1];
            ck.plane[a.nz + z] = v[2];
            // next reference: the plane mean of T on the quantum grid
            ck.rc[z] = (float)(nearbyint(v[3] * ck.inv_area * ck.inv_quantum) * ck.quantum);
            ck.plane_cnt[z] = 0;
            __threadfence();
            const unsigned ticket = atomicAdd(&ck.ctl->glob_cnt, 1u);
            s_last_plane = ticket == (unsigned)a.nz - 1u;
        }
    }
    __syncthreads();
    if (s_last_plane) {
        __threadfence();
        close_check(a);
    }
}

// One fused pull-stream + collide step over 4 consecutive voxels of a row per
// thread.  Threads of a block cover consecutive quads of one z-plane, so the
// x-neighbours of a quad sit in the adjacent lanes (warp shuffles) except at
// warp and row boundaries, where a scalar load or a face rule supplies them.
template <bool PERIODIC, bool CHECK>
__global__ void __launch_bounds__(kThreads) step_kernel(const StepArgs a) {
    extern __shared__ float4 s_sb[];
    for (int i = threadIdx.x; i < 2 * a.n_phases; i += kThreads) s_sb[i] = a.sb[i];
    __syncthreads();

    const int nq = a.pitch >> 2;
    const int t = blockIdx.x * kThreads + threadIdx.x;    // quad index within the plane
    const int z = blockIdx.y;
    const bool active = t < a.quads_per_plane;
    const int y = active ? t / nq : 0;
    const int qx = active ? t - y * nq : 0;
    const int x0 = qx << 2;
    const int lane = threadIdx.x & 31;
    const long long P = a.pstride;
    const float* __restrict__ src = a.src;

    const long long row = ((long long)z * a.ny + y) * a.pitch;
    // y-neighbour rows: periodic wrap (Eq. 25) or bounce-back into the own node (Eq. 24)
    const bool ylo = (y == 0), yhi = (y == a.ny - 1);
    const bool zlo = (z == 0), zhi = (z == a.nz - 1);
    const long long rym = PERIODIC ? ((long long)z * a.ny + (ylo ? a.ny - 1 : y - 1)) * a.pitch
                                   : (ylo ? row + 4 * P : row - a.pitch + 3 * P);
    const long long ryp = PERIODIC ? ((long long)z * a.ny + (yhi ? 0 : y + 1)) * a.pitch
                                   : (yhi ? row + 3 * P : row + a.pitch + 4 * P);
    const long long o3 = PERIODIC ? rym + 3 * P : rym;
    const long long o4 = PERIODIC ? ryp + 4 * P : ryp;
    // z-neighbour rows; the walls (Eq. 23) read the own node's opposite population
    const long long o5 = zlo ? row + 6 * P : row - (long long)a.ny * a.pitch + 5 * P;
    const long long o6 = zhi ? row + 5 * P : row + (long long)a.ny * a.pitch + 6 * P;

    float4 c0 = make_float4(0.f, 0.f, 0.f, 0.f), c1 = c0, c2 = c0, c3 = c0, c4 = c0, c5 = c0, c6 = c0;
    uchar4 ph = make_uchar4(0, 0, 0, 0);
    if (active) {
        c0 = ld4(src + row + x0);
        c1 = ld4(src + P + row + x0);
        c2 = ld4(src + 2 * P + row + x0);
        c3 = ld4(src + o3 + x0);
        c4 = ld4(src + o4 + x0);
        c5 = ld4(src + o5 + x0);
        c6 = ld4(src + o6 + x0);
        ph = __ldg(reinterpret_cast<const uchar4*>(a.phase + row + x0));
    }
    // Frame changes (all exact): a population pulled from plane z' carries
    // w_i R_src(z'); it is re-expressed relative to R_dst(z) of this node.
    const float w = 0.125f;
    const float r0 = a.rsrc[z], rd = a.rdst[z];
    const float rm = zlo ? r0 : a.rsrc[z - 1];
    const float rp = zhi ? r0 : a.rsrc[z + 1];
    const float k_in = w * (r0 - rd);
    // walls (Eq. 23): f_in = -fhat_out(x) + eps T_wall, fhat_out = g + w R_src(z)
    const float k5 = zlo ? (a.eps_hot - w * r0) - w * rd : w * (rm - rd);
    const float k6 = zhi ? (a.eps_cold - w * r0) - w * rd : w * (rp - rd);
    const float kT = (2.f * k_in + 4.f * k_in) + (k5 + k6);   // sum of w_i (...) with w_0 = 2w
    const float kJ = k5 - k6;
    if (zlo) { c5.x = -c5.x; c5.y = -c5.y; c5.z = -c5.z; c5.w = -c5.w; }
    if (zhi) { c6.x = -c6.x; c6.y = -c6.y; c6.z = -c6.z; c6.w = -c6.w; }
    // x-neighbours: f1 comes from x - 1, f2 from x + 1.
    const float left1 = __shfl_up_sync(kFull, c1.w, 1);
    const float right2 = __shfl_down_sync(kFull, c2.x, 1);
    float4 f1, f2;
    f1.y = c1.x; f1.z = c1.y; f1.w = c1.z;
    f2.x = c2.y; f2.y = c2.z; f2.z = c2.w;
    if (lane > 0 && qx > 0) f1.x = left1;
    else if (qx > 0) f1.x = active ? __ldg(src + P + row + x0 - 1) : 0.f;
    else f1.x = PERIODIC ? (active ? __ldg(src + P + row + a.nx - 1) : 0.f) : c2.x;
    if (qx < nq - 1) {
        f2.w = (lane < 31) ? right2 : (active ? __ldg(src + 2 * P + row + x0 + 4) : 0.f);
    } else {
        f2.w = 0.f;
        // the last real voxel of the row sits in this quad
        const int e = a.nx - 1 - x0;
        const float edge = PERIODIC ? (active ? __ldg(src + 2 * P + row) : 0.f) : comp(c1, e);
        set_comp(f2, e, edge);
    }

    const int n_real = active ? min(4, a.nx - x0) : 0;
    float4 o0v, o1v, o2v, o3v, o4v, o5v, o6v;
    float4 thv, thp = make_float4(0.f, 0.f, 0.f, 0.f);
    // per-thread (4 voxels) and per-warp sums of positive FP32 terms stay in
    // FP32; the block tree, the plane sums and the residual sums are FP64
    float q_sum = 0.f, dT_sum = 0.f, T_sum = 0.f, Tp_sum = 0.f;
    // T - T_ref at the previous check: the residual is the change since then
    if (CHECK && active) thp = *reinterpret_cast<const float4*>(a.tsnap + row + x0);
    const float dref = (float)((double)rd - a.t_ref);
    const float tref = (float)a.t_ref;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float g0 = comp(c0, k), g1 = comp(f1, k), g2 = comp(f2, k), g3 = comp(c3, k);
        const float g4 = comp(c4, k), g5 = comp(c5, k), g6 = comp(c6, k);
        const int p = (k == 0 ? ph.x : (k == 1 ? ph.y : (k == 2 ? ph.z : ph.w)));
        const float4 sa = s_sb[2 * p];
        const float4 sc = s_sb[2 * p + 1];
        // T - R_dst(z) (Eq. 14) and the flux moment j, with the frame constants
        const float th = (((g0 + g1) + (g2 + g3)) + ((g4 + g5) + g6)) + kT;
        const float jx = g1 - g2, jy = g3 - g4, jz = (g5 - g6) + kJ;
        // sigma = S_b j with S_b symmetric: (xx, yy, zz, yz) = sa, (xz, xy) = sc.xy
        const float sx = fmaf(sa.x, jx, fmaf(sc.y, jy, sc.x * jz));
        const float sy = fmaf(sc.y, jx, fmaf(sa.y, jy, sa.w * jz));
        const float sz = fmaf(sc.x, jx, fmaf(sa.w, jy, sa.z * jz));
        const float hx = jx - sx, hy = jy - sy, hz = jz - sz;
        const float t8 = 0.125f * th;
        const bool real = k < n_real;
        set_comp(o0v, k, real ? 0.25f * th : 0.f);
        set_comp(o1v, k, real ? fmaf(0.5f, hx, t8) : 0.f);
        set_comp(o2v, k, real ? fmaf(-0.5f, hx, t8) : 0.f);
        set_comp(o3v, k, real ? fmaf(0.5f, hy, t8) : 0.f);
        set_comp(o4v, k, real ? fmaf(-0.5f, hy, t8) : 0.f);
        set_comp(o5v, k, real ? fmaf(0.5f, hz, t8) : 0.f);
        set_comp(o6v, k, real ? fmaf(-0.5f, hz, t8) : 0.f);
        if (CHECK) {
            const float tdev = th + dref;                    // T - T_ref
            set_comp(thv, k, real ? tdev : 0.f);
            if (real) {
                q_sum += fmaf(-0.5f, sz, jz);                // (j_z + jhat_z) / 2
                dT_sum += fabsf(tdev - comp(thp, k));
                T_sum += fabsf(tdev + tref);
                Tp_sum += tdev + tref;
            }
        }
    }
    if (active) {
        float* __restrict__ dst = a.dst + row + x0;
        st4(dst, o0v);
        st4(dst + P, o1v);
        st4(dst + 2 * P, o2v);
        st4(dst + 3 * P, o3v);
        st4(dst + 4 * P, o4v);
        st4(dst + 5 * P, o5v);
        st4(dst + 6 * P, o6v);
        if (CHECK) st4(a.tsnap + row + x0, thv);
    }

    if (CHECK) {
        // warp shuffle, then a tree over the block's warps: one FP64 partial
        // per (block, plane) written in a fixed order (deterministic)
        float vf[4] = {q_sum, dT_sum, T_sum, Tp_sum};
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int m = 0; m < 4; ++m) vf[m] += __shfl_down_sync(kFull, vf[m], off);
        double v[4];
        __shared__ double s_red[4][kThreads / 32];
        __shared__ int s_last;
        const int warp = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int m = 0; m < 4; ++m) s_red[m][warp] = (double)vf[m];
        __syncthreads();
        if (threadIdx.x < 32) {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = lane < kThreads / 32 ? s_red[m][lane] : 0.0;
#pragma unroll
            for (int off = 4; off > 0; off >>= 1)
#pragma unroll
                for (int m = 0; m < 4; ++m) v[m] += __shfl_down_sync(kFull, v[m], off);
            if (lane == 0) {
                const CheckArgs& ck = a.ck;
                const long long base = (long long)z * a.blocks_per_plane + blockIdx.x;
                const long long plane_all = (long long)a.nz * a.blocks_per_plane;
#pragma unroll
                for (int m = 0; m < 4; ++m) ck.part[m * plane_all + base] = v[m];
                // the last block of this plane to finish closes the plane
                __threadfence();
                const int ticket = atomicAdd(&ck.plane_cnt[z], 1);
                s_last = ticket == a.blocks_per_plane - 1;
            }
        }
        __syncthreads();
        if (s_last) close_plane(a, z);
    }
}

__global__ void add_iters_kernel(Ctl* c, long long n) { c->iter += n; }

// Canonical layout: new axis i is old axis perm[i]; rows padded to pitch.
struct Layout {
    int n[3];          // original nx, ny, nz
    int perm[3];
    int NX, NY, NZ, pitch;
};

__device__ __forceinline__ long long orig_index(const Layout& L, int xc, int yc, int zc) {
    int c[3];
    c[L.perm[0]] = xc;
    c[L.perm[1]] = yc;
    c[L.perm[2]] = zc;
    return ((long long)c[2] * L.n[1] + c[1]) * L.n[0] + c[0];
}

// Gathers the phase map into the canonical padded layout.
__global__ void permute_phase_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, Layout L) {
    const long long total = (long long)L.pitch * L.NY * L.NZ;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int xc = (int)(i % L.pitch);
        const long long r = i / L.pitch;
        const int yc = (int)(r % L.NY);
        const int zc = (int)(r / L.NY);
        out[i] = xc < L.NX ? in[orig_index(L, xc, yc, zc)] : (uint8_t)0;
    }
}

// Initial state fhat^0 = f^eq(T0) (Eq. 6) as deviations from w_i T_ref.
// T0 is the linear profile between the walls, or a given field (original order).
// plane_th[z] = T0(z) - R(z) and plane_ts[z] = T0(z) - T_ref for the linear
// start (host FP64, rounded once); a caller field t_init replaces T0.
__global__ void init_kernel(float* __restrict__ f, float* __restrict__ tsnap, long long P, Layout L,
                            const float* __restrict__ ref, const float* __restrict__ plane_th,
                            const float* __restrict__ plane_ts, float t_ref,
                            const float* __restrict__ t_init) {
    const long long total = (long long)L.pitch * L.NY * L.NZ;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int xc = (int)(i % L.pitch);
        const long long r = i / L.pitch;
        const int yc = (int)(r % L.NY);
        const int zc = (int)(r / L.NY);
        float th = 0.f, ts = 0.f;
        if (xc < L.NX) {
            if (t_init) {
                const float T = t_init[orig_index(L, xc, yc, zc)];
                th = T - ref[zc];
                ts = T - t_ref;
            } else {
                th = plane_th[zc];
                ts = plane_ts[zc];
            }
        }
        tsnap[i] = ts;
        f[i] = 0.25f * th;
        const float e = 0.125f * th;
        for (int q = 1; q < 7; ++q) f[q * P + i] = e;
    }
}

// T = sum_i f_i (Eq. 14) of the current state, written in the original order.
__global__ void temperature_kernel(const float* __restrict__ f, long long P, Layout L,
                                   const float* __restrict__ ref, float* __restrict__ T) {
    const long long total = (long long)L.n[0] * L.n[1] * L.n[2];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        int c[3];
        c[0] = (int)(i % L.n[0]);
        const long long r = i / L.n[0];
        c[1] = (int)(r % L.n[1]);
        c[2] = (int)(r / L.n[1]);
        const int zc = c[L.perm[2]];
        const long long k = ((long long)zc * L.NY + c[L.perm[1]]) * L.pitch + c[L.perm[0]];
        const float th = ((f[k] + f[P + k]) + (f[2 * P + k] + f[3 * P + k])) +
                         ((f[4 * P + k] + f[5 * P + k]) + f[6 * P + k]);
        T[i] = th + ref[zc];
    }
}

}  // namespace lbm
