// Device kernels of the D3Q7 MRT lattice Boltzmann hot path for sm_103a.
//
// Storage: the post-collision state of every node lies in a four-dimensional
// subspace (see the collision below: fhat_0 = T / 4, fhat_{2k-1,2k} = T / 8 +-
// jhat_k / 2), so the state is stored as four fields per node, th = T - R(z)
// and m = jhat / 2, not seven populations: structure of arrays
// [field][z][y][x], FP32, BF16 or FP16, two buffers (pull scheme: read the
// previous post-collision state, write the next one).  A node rebuilds each
// population it pulls from its source node's fields (f_{2k-1} = th / 8 + m_k,
// f_{2k} = th / 8 - m_k, f_0 = th / 4); the scalings by 1/8 and 1/4 are exact,
// so in FP32 the pulled values are the very populations a seven-field state
// would have stored, while a step moves 16 instead of 28 bytes per node.  The
// Dirichlet axis is always the slowest index z; the host lays the cell out
// that way.  Rows are padded to a multiple of V voxels (pitch) so that every
// thread moves one aligned 16-byte vector per field (V = 4 FP32 or 8 16-bit
// values).
// The temperature is stored as the deviation th = T - R(z) from a per-plane
// reference temperature R(z) (populations g_i = f_i - w_i R(z), w_0 = 1/4,
// w_1..6 = 1/8, Eq. 6 with gamma = 1/8): the plane mean of T at the previous
// check, quantised to a power-of-two grid so that every frame-change constant
// w_i (R(z') - R(z)) is exact in FP32.  The map is linear, so the frame
// changes nothing in exact arithmetic; in FP32 the stored values are small
// (non-equilibrium parts and in-plane temperature variation), which shrinks
// the rounding of the stored state and with it the FP32 error of the
// converged fixed point.
//
// Collision (Eq. 5, 8-13).  With tau_0 = tau_4 = tau_5 = tau_6 = 1 the
// moments 0, 4, 5, 6 leave the collision at equilibrium and the flux moment
// j = (f1 - f2, f3 - f4, f5 - f6) relaxes to jhat = j - S_b j with
// S_b = tau^-1 (the 3x3 off-diagonal block of Eq. 12 inverted).  Because the
// rows of M in Eq. 11 are orthogonal, M^-1 maps this back to
//   fhat_0 = T / 4,   fhat_{2k-1,2k} = T / 8 +- jhat_k / 2,
// which is M^-1 S M applied exactly (no 7x7 product on the device).  The
// device holds, per phase, the symmetric B = (I - S_b) / 2, so jhat_k / 2 =
// (B j)_k: one 3x3 product and no further scaling per node.
// Interfaces need no code: each node uses its own phase's table entry and
// streaming is plain (Eq. 21, the half-lattice division scheme of Section 2.3).
//
// Flux (Eq. 15-16).  With D = eps (tau - I/2) and grad T = -tau^-1 j / eps,
// q = -D grad T = (I - S_b / 2) j = (j + jhat) / 2 = j / 2 + B j at every node.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

namespace lbm {

// Bounds-checked build (-DLBM_DEBUG, `build.build(debug=True)`): every
// global and ring access of the step kernels is checked against its buffer;
// an access outside records its code in the device word g_lbm_debug (one per
// translation unit) and goes to the buffer's first element instead.  The host
// calls turn a recorded code into LBM_ERR_INTERNAL.  This stands in for a
// memory checker: the index arithmetic of every launch is checked while the
// parity tests run.  Without LBM_DEBUG the checks compile to nothing.
#ifdef LBM_DEBUG
static __device__ unsigned int g_lbm_debug = 0u;
template <typename T>
__device__ __forceinline__ T* dbg_ptr(T* p, T* base, long long count, int width, unsigned code) {
    const long long i = p - base;
    if (i < 0 || i + width > count) {
        atomicCAS(&g_lbm_debug, 0u, code);
        return base;
    }
    return p;
}
#define LBM_CK(p, base, count, width, code) ::lbm::dbg_ptr((p), (base), (long long)(count), (width), (code))
#else
#define LBM_CK(p, base, count, width, code) (p)
#endif

constexpr int kThreads = 256;        // threads per step block
constexpr int kFields = 4;           // stored fields per node: th, m_x, m_y, m_z
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
    double* hist;                    // history ring [hist_cap][4] or null
    unsigned long long* hist_t;      // device time (ns) of each history row, or null
    int hist_cap;
};

struct StepArgs {
    const void* __restrict__ src;    // fields th, m_x, m_y, m_z of post-collision state n-1
    void* __restrict__ dst;          // the fields of post-collision state n
    const uint8_t* __restrict__ phase;  // [nz][ny][pitch], padded with 0
    const float4* __restrict__ sb;   // 2 float4 per phase: (xx, yy, zz, yz), (xz, xy, -, -)
    float* __restrict__ tsnap;       // T - T_ref at the previous check, [nz][ny][pitch]
    const float* __restrict__ rsrc;  // reference R(z) of the src state, [nz]
    const float* __restrict__ rdst;  // reference R(z) of the dst state, [nz]
    long long pstride;               // elements per field = pitch * ny * nz
    int nx, ny, nz, pitch, n_phases;
    int quads_per_plane;             // (pitch / V) * ny vectors per plane
    int blocks_per_plane;
    int zrev;                        // 1: blocks walk the planes from the top (alternate steps)
    float eps_hot, eps_cold;         // eps * T_wall
    unsigned rseed;                  // launch salt of the stochastic rounding
    int f2_fy, f2_bxy, f2_zchunk;    // two-step tiles of this solve in a batch launch
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

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Closing a check (Eq. 15-16 plane sums, Eq. 22, the stop rule).  Every
// block of a check step writes its FP64 partials and takes a ticket on its
// plane's counter; the block that takes the last ticket sums the plane's
// partials in block order, and the block that closes the last plane sums the
// planes in plane order and applies the stop rule.  No block ever waits:
// the work falls to whichever block finishes last, and the result is
// deterministic.

template <int THREADS>
__device__ void close_check(const StepArgs& a) {
    const CheckArgs& ck = a.ck;
    double qsum = 0.0, qmax = -INFINITY, qmin = INFINITY, dsum = 0.0, tsum = 0.0;
    for (int z = threadIdx.x; z < a.nz; z += THREADS) {
        const double q = __ldcg(ck.Q + z);
        qsum += q;
        qmax = fmax(qmax, q);
        qmin = fmin(qmin, q);
        dsum += __ldcg(ck.plane + z);
        tsum += __ldcg(ck.plane + a.nz + z);
    }
    __shared__ double s[5][THREADS / 32];
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
    for (int z = threadIdx.x; z < a.nz; z += THREADS) {
        if (ck.rebase) ck.ra[z] = ck.rb[z];
        ck.rb[z] = __ldcg(ck.rc + z);
    }
    if (threadIdx.x == 0) {
        qsum = 0.0; qmax = -INFINITY; qmin = INFINITY; dsum = 0.0; tsum = 0.0;
        for (int w = 0; w < THREADS / 32; ++w) {
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
        if (ck.hist_t) ck.hist_t[(c->checks - 1) % ck.hist_cap] = globaltimer_ns();
        if (ck.hist) {
            double* hrow = ck.hist + 4 * ((c->checks - 1) % ck.hist_cap);
            hrow[0] = (double)c->iter;
            hrow[1] = c->k_eff;
            hrow[2] = c->r_t;
            hrow[3] = c->r_q;
        }
        const bool stop = status != 5 || c->iter + ck.interval > ck.max_iters;
        c->done = stop ? 1 : 0;
        c->glob_cnt = 0u;
        if (ck.use_handle) cudaGraphSetConditional(ck.handle, stop ? 0u : 1u);
    }
}

template <int THREADS>
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
        close_check<THREADS>(a);
    }
}

// The collision of one node (Eq. 5, 8-13 in the reduced form above) from its
// seven pulled values relative to R_src, with the frame constants kT, kJ and
// the phase's table entry (sa, sc) = B; returns the fields the
// state stores, th = T - R_dst and m = jhat / 2, and q_z, the flux along z
// (Eq. 16).  Every step kernel uses this one function.
struct Collided {
    float th;
    float m[3];
    float qz;
};

// host side of the table: the entry of one phase, B = (I - S_b) / 2 from S_b
// (FP64, 3x3 row-major), rounded once to FP32
inline void phase_entry(const double* S, float4* e) {
    e[0] = make_float4((float)(0.5 * (1.0 - S[0])), (float)(0.5 * (1.0 - S[4])),
                       (float)(0.5 * (1.0 - S[8])), (float)(-0.5 * S[5]));
    e[1] = make_float4((float)(-0.5 * S[2]), (float)(-0.5 * S[1]), 0.f, 0.f);
}

__device__ __forceinline__ Collided collide_node(float g0, float g1, float g2, float g3, float g4,
                                                 float g5, float g6, float4 sa, float4 sc, float kT,
                                                 float kJ) {
    Collided c;
    // T - R_dst(z) (Eq. 14) and the flux moment j, with the frame constants
    c.th = (((g0 + g1) + (g2 + g3)) + ((g4 + g5) + g6)) + kT;
    const float jx = g1 - g2, jy = g3 - g4, jz = (g5 - g6) + kJ;
    // a = B j = jhat / 2 with the symmetric B: (xx, yy, zz, yz) = sa, (xz, xy) = sc.xy
    c.m[0] = fmaf(sa.x, jx, fmaf(sc.y, jy, sc.x * jz));
    c.m[1] = fmaf(sc.y, jx, fmaf(sa.y, jy, sa.w * jz));
    c.m[2] = fmaf(sc.x, jx, fmaf(sa.w, jy, sa.z * jz));
    c.qz = fmaf(0.5f, jz, c.m[2]);      // j_z / 2 + (B j)_z
    return c;
}

// A post-collision population from the stored fields of the node it leaves:
// f_{2k-1} = th / 8 + m_k (pull_p) and f_{2k} = th / 8 - m_k (pull_m), the
// rest population f_0 = th / 4.  The scalings are exact, so each value is
// the population the collision would have stored, rounded once.
__device__ __forceinline__ float pull_p(float th, float m) { return fmaf(0.125f, th, m); }
__device__ __forceinline__ float pull_m(float th, float m) { return fmaf(0.125f, th, -m); }

// Frame constants of plane z for a step from frame R_src to R_dst (see the
// step kernel): kT is added to the sum of the pulled values, kJ to j_z.
struct PlaneK {
    float kT, kJ;
};

__device__ __forceinline__ PlaneK plane_consts(const float* rsrc, const float* rdst, int z, int nz,
                                               float eps_hot, float eps_cold) {
    const float w = 0.125f;
    const bool zlo = z == 0, zhi = z == nz - 1;
    const float r0 = rsrc[z], rd = rdst[z];
    const float rm = zlo ? r0 : rsrc[z - 1];
    const float rp = zhi ? r0 : rsrc[z + 1];
    const float k_in = w * (r0 - rd);
    const float k5 = zlo ? (eps_hot - w * r0) - w * rd : w * (rm - rd);
    const float k6 = zhi ? (eps_cold - w * r0) - w * rd : w * (rp - rd);
    PlaneK k;
    k.kT = (2.f * k_in + 4.f * k_in) + (k5 + k6);
    k.kJ = k5 - k6;
    return k;
}

// Storage policies.  FP32 moves 4 voxels per thread as one float4 per
// field; BF16 and FP16 move 8 voxels per thread as one uint4 (eight 16-bit
// values) per field, converted to FP32 for the collision and
// rounded back stochastically (cvt.rs: the rounding direction is drawn with
// probability proportional to the distance to each neighbour, so the stored
// value is unbiased and updates below half an ulp are not lost on average).
template <int FMT> struct Pol;

template <> struct Pol<0> {
    using T = float;
    using Raw = float4;
    static constexpr int V = 4;
    __device__ static Raw zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    __device__ static Raw load(const T* p) { return ld4(p); }
    __device__ static float get(const Raw& r, int k) { return comp(r, k); }
    __device__ static float scalar(const T* p) { return __ldg(p); }
    __device__ static Raw neg(Raw r) { return make_float4(-r.x, -r.y, -r.z, -r.w); }
    __device__ static void store(T* p, const float (&o)[V], unsigned) {
        st4(p, make_float4(o[0], o[1], o[2], o[3]));
    }
};

__device__ __forceinline__ unsigned word(const uint4& r, int m) {
    return m == 0 ? r.x : (m == 1 ? r.y : (m == 2 ? r.z : r.w));
}

__device__ __forceinline__ unsigned hash32(unsigned x) {   // lowbias32 (C. Wellons)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int FMT> struct Pol16 {
    using T = uint16_t;
    using Raw = uint4;
    static constexpr int V = 8;
    __device__ static Raw zero() { return make_uint4(0u, 0u, 0u, 0u); }
    __device__ static Raw load(const T* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }
    __device__ static float from16(unsigned h) {
        if (FMT == 1) return __uint_as_float(h << 16);                  // bf16
        return __half2float(__ushort_as_half((unsigned short)h));       // fp16
    }
    __device__ static float get(const Raw& r, int k) {
        const unsigned w = word(r, k >> 1);
        return from16((k & 1) ? (w >> 16) : (w & 0xffffu));
    }
    __device__ static float scalar(const T* p) { return from16(__ldg(p)); }
    __device__ static Raw neg(Raw r) {
        return make_uint4(r.x ^ 0x80008000u, r.y ^ 0x80008000u, r.z ^ 0x80008000u, r.w ^ 0x80008000u);
    }
    // pairs (o[2m], o[2m+1]) -> low and high half of word m; rbits[31:16]
    // round the high half, rbits[15:0] the low half
    __device__ static unsigned pack(float lo, float hi, unsigned rbits) {
        unsigned d;
        if (FMT == 1)
            asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
        else
            asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
        return d;
    }
    // one hash per vector; the four words are distinct affine maps of it
    // (each uniform on its own, which is all an unbiased rounding needs)
    __device__ static void store(T* p, const float (&o)[V], unsigned key) {
        const unsigned h = hash32(key);
        uint4 r;
        r.x = pack(o[0], o[1], h);
        r.y = pack(o[2], o[3], h * 0x2C1B3C6Du + 0x297A2D39u);
        r.z = pack(o[4], o[5], h * 0x85EBCA6Bu + 0x68E31DA4u);
        r.w = pack(o[6], o[7], h * 0xCC9E2D51u + 0x1B873593u);
        *reinterpret_cast<uint4*>(p) = r;
    }
};
template <> struct Pol<1> : Pol16<1> {};
template <> struct Pol<2> : Pol16<2> {};

// One fused pull-stream + collide step over V consecutive voxels of a row per
// thread (V = 4 in FP32, 8 in 16-bit storage).  Threads of a block cover
// consecutive vectors of one z-plane, so the x-neighbours of a vector sit in
// the adjacent lanes (warp shuffles) except at warp and row boundaries, where
// a scalar load or a face rule supplies them.  RAGGED: nx is not a multiple
// of V, so the last vector of a row holds padding.
// A node pulls f_i from its neighbour at -e_i, rebuilt from that node's
// stored fields: th and m_x of the x-neighbours, th and m_y of the
// y-neighbours, th and m_z of the z-neighbours, th of the own node.
template <int FMT, bool PERIODIC, bool CHECK, bool RAGGED, int THREADS>
__device__ __forceinline__ void step_body(const StepArgs& a, const int bx, const int z,
                                          const unsigned rseed) {
    using S = Pol<FMT>;
    using T = typename S::T;
    using Raw = typename S::Raw;
    constexpr int V = S::V;
    extern __shared__ float4 s_sb[];
    for (int i = threadIdx.x; i < 2 * a.n_phases; i += THREADS) s_sb[i] = a.sb[i];
    __syncthreads();

    const int nq = a.pitch / V;
    const int t = bx * THREADS + threadIdx.x;             // vector index within the plane
    const bool active = t < a.quads_per_plane;
    const int y = active ? t / nq : 0;
    const int qx = active ? t - y * nq : 0;
    const int x0 = qx * V;
    const int lane = threadIdx.x & 31;
    const long long P = a.pstride;
    const long long PL = (long long)a.ny * a.pitch;
    const T* __restrict__ src = reinterpret_cast<const T*>(a.src);
    constexpr int NF = kFields;

    const long long row = ((long long)z * a.ny + y) * a.pitch;
    // y-neighbour rows: periodic wrap (Eq. 25), or the own node at an
    // adiabatic face (bounce-back, Eq. 24: m_y enters with the other sign)
    const bool ylo = (y == 0), yhi = (y == a.ny - 1);
    const bool zlo = (z == 0), zhi = (z == a.nz - 1);
    const long long rym = ylo ? (PERIODIC ? row + (long long)(a.ny - 1) * a.pitch : row) : row - a.pitch;
    const long long ryp = yhi ? (PERIODIC ? row - (long long)(a.ny - 1) * a.pitch : row) : row + a.pitch;
    // z-neighbour planes; the walls (Eq. 23) use the own node, th with the
    // other sign (anti-bounce-back)
    const long long rzm = zlo ? row : row - PL;
    const long long rzp = zhi ? row : row + PL;

    // a thread past the plane's last vector (active false) loads row 0 of
    // the plane: in bounds, and nothing it computes is stored or summed
    Raw cT, cX, mT, mY, pT, pY, dT, dZ, uT, uZ;
    uint2 ph = make_uint2(0u, 0u);
    {
        cT = S::load(LBM_CK(src + row + x0, src, NF * P, V, 1u));
        cX = S::load(LBM_CK(src + P + row + x0, src, NF * P, V, 1u));
        mT = S::load(LBM_CK(src + rym + x0, src, NF * P, V, 1u));
        mY = S::load(LBM_CK(src + 2 * P + rym + x0, src, NF * P, V, 1u));
        pT = S::load(LBM_CK(src + ryp + x0, src, NF * P, V, 1u));
        pY = S::load(LBM_CK(src + 2 * P + ryp + x0, src, NF * P, V, 1u));
        dT = S::load(LBM_CK(src + rzm + x0, src, NF * P, V, 1u));
        dZ = S::load(LBM_CK(src + 3 * P + rzm + x0, src, NF * P, V, 1u));
        uT = S::load(LBM_CK(src + rzp + x0, src, NF * P, V, 1u));
        uZ = S::load(LBM_CK(src + 3 * P + rzp + x0, src, NF * P, V, 1u));
        if (V == 8) ph = __ldg(reinterpret_cast<const uint2*>(LBM_CK(a.phase + row + x0, a.phase, P, V, 2u)));
        else ph.x = __ldg(reinterpret_cast<const unsigned*>(LBM_CK(a.phase + row + x0, a.phase, P, V, 2u)));
    }
    // Frame changes (all exact): a population pulled from plane z' carries
    // w_i R_src(z'); it is re-expressed relative to R_dst(z) of this node.
    const PlaneK pk = plane_consts(a.rsrc, a.rdst, z, a.nz, a.eps_hot, a.eps_cold);
    const float kT = pk.kT, kJ = pk.kJ;
    const float rd = a.rdst[z];
    if (zlo) dT = S::neg(dT);
    if (zhi) uT = S::neg(uT);
    if (!PERIODIC && ylo) mY = S::neg(mY);
    if (!PERIODIC && yhi) pY = S::neg(pY);
    // x-neighbours: f1 comes from x - 1, f2 from x + 1 (th and m_x of each)
    const float lT = __shfl_up_sync(kFull, S::get(cT, V - 1), 1);
    const float lX = __shfl_up_sync(kFull, S::get(cX, V - 1), 1);
    const float rT = __shfl_down_sync(kFull, S::get(cT, 0), 1);
    const float rX = __shfl_down_sync(kFull, S::get(cX, 0), 1);
    float TL, XL, TR, XR;
    if (lane > 0 && qx > 0) {
        TL = lT;
        XL = lX;
    } else if (qx > 0 || PERIODIC) {
        const long long xl = qx > 0 ? row + x0 - 1 : row + a.nx - 1;
        TL = active ? S::scalar(LBM_CK(src + xl, src, NF * P, 1, 3u)) : 0.f;
        XL = active ? S::scalar(LBM_CK(src + P + xl, src, NF * P, 1, 3u)) : 0.f;
    } else {                                      // Eq. 24 at x = 0: f1 = f2 of the own node
        TL = S::get(cT, 0);
        XL = -S::get(cX, 0);
    }
    // the last real voxel of the row sits in the row's last vector, at e_last
    const int e_last = (RAGGED && qx == nq - 1) ? a.nx - 1 - x0 : V;
    float eT = 0.f, eX = 0.f;
    if (qx < nq - 1) {
        if (lane < 31) {
            TR = rT;
            XR = rX;
        } else {
            TR = active ? S::scalar(LBM_CK(src + row + x0 + V, src, NF * P, 1, 3u)) : 0.f;
            XR = active ? S::scalar(LBM_CK(src + P + row + x0 + V, src, NF * P, 1, 3u)) : 0.f;
        }
    } else {
        if (PERIODIC) {                           // the row's first node
            eT = active ? S::scalar(LBM_CK(src + row, src, NF * P, 1, 3u)) : 0.f;
            eX = active ? S::scalar(LBM_CK(src + P + row, src, NF * P, 1, 3u)) : 0.f;
        } else {                                  // Eq. 24 at x = nx - 1: f2 = f1 of the own node
            eT = S::get(cT, V - 1);
            eX = -S::get(cX, V - 1);
        }
        TR = RAGGED ? 0.f : eT;
        XR = RAGGED ? 0.f : eX;
    }

    const int n_real = active ? min(V, a.nx - x0) : 0;
    // per-thread and per-warp sums of positive FP32 terms stay in FP32; the
    // block tree, the plane sums and the residual sums are FP64
    float q_sum = 0.f, dT_sum = 0.f, T_sum = 0.f, Tp_sum = 0.f;
    float thp[V], thv[V];
    // T - T_ref at the previous check: the residual is the change since then
    if (CHECK) {
#pragma unroll
        for (int v4 = 0; v4 < V / 4; ++v4) {
            const float4 q4 = active ? *reinterpret_cast<const float4*>(LBM_CK(a.tsnap + row + x0 + 4 * v4, a.tsnap, P, 4, 4u))
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
            thp[4 * v4] = q4.x; thp[4 * v4 + 1] = q4.y; thp[4 * v4 + 2] = q4.z; thp[4 * v4 + 3] = q4.w;
        }
    }
    const float dref = (float)((double)rd - a.t_ref);
    const float tref = (float)a.t_ref;
    float o[NF][V];
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const float g0 = 0.25f * S::get(cT, k);
        const float g1 = k == 0 ? pull_p(TL, XL) : pull_p(S::get(cT, k - 1), S::get(cX, k - 1));
        float g2 = k == V - 1 ? pull_m(TR, XR) : pull_m(S::get(cT, k + 1), S::get(cX, k + 1));
        if (RAGGED && k == e_last) g2 = PERIODIC ? pull_m(eT, eX) : pull_p(S::get(cT, k), S::get(cX, k));
        const float g3 = pull_p(S::get(mT, k), S::get(mY, k)), g4 = pull_m(S::get(pT, k), S::get(pY, k));
        const float g5 = pull_p(S::get(dT, k), S::get(dZ, k)), g6 = pull_m(S::get(uT, k), S::get(uZ, k));
        const int p = (k < 4 ? (ph.x >> (8 * k)) : (ph.y >> (8 * (k - 4)))) & 0xff;
        const float4 sa = s_sb[2 * p];
        const float4 sc = s_sb[2 * p + 1];
        const Collided cc = collide_node(g0, g1, g2, g3, g4, g5, g6, sa, sc, kT, kJ);
        const float th = cc.th;
        const bool real = RAGGED ? k < n_real : active;   // n_real is 0 for inactive threads
        o[0][k] = th;
        o[1][k] = cc.m[0];
        o[2][k] = cc.m[1];
        o[3][k] = cc.m[2];
        if (CHECK) {
            const float tdev = th + dref;                    // T - T_ref
            thv[k] = tdev;
            if (real) {
                q_sum += cc.qz;                              // (j_z + jhat_z) / 2
                dT_sum += fabsf(tdev - thp[k]);
                T_sum += fabsf(tdev + tref);
                Tp_sum += tdev + tref;
            }
        }
    }
    if (RAGGED && n_real < V) {
        // padding voxels of the row's last vector stay zero
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (k >= n_real) {
#pragma unroll
                for (int i = 0; i < NF; ++i) o[i][k] = 0.f;
                if (CHECK) thv[k] = 0.f;
            }
    }
    if (active) {
        T* __restrict__ dst = reinterpret_cast<T*>(a.dst) + row + x0;
        // random bits for stochastic rounding: a hash of the element's
        // position and field, salted by the iteration and the launch
        unsigned key = 0u;
        if (FMT != 0) {
            const unsigned seed = hash32((unsigned)__ldcg(&a.ck.ctl->iter) * 0x9E3779B9u + rseed);
            key = seed ^ (unsigned)((row + x0) >> 1) * 0x85ebca6bu;
        }
#pragma unroll
        for (int i = 0; i < NF; ++i)
            S::store(LBM_CK(dst + i * P, reinterpret_cast<T*>(a.dst), NF * P, V, 5u), o[i], key + 0x9E3779B9u * (unsigned)i);
        if (CHECK) {
#pragma unroll
            for (int v4 = 0; v4 < V / 4; ++v4)
                st4(LBM_CK(a.tsnap + row + x0 + 4 * v4, a.tsnap, P, 4, 4u),
                    make_float4(thv[4 * v4], thv[4 * v4 + 1], thv[4 * v4 + 2], thv[4 * v4 + 3]));
        }
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
        __shared__ double s_red[4][THREADS / 32];
        __shared__ int s_last;
        const int warp = threadIdx.x >> 5;
        if (lane == 0)
#pragma unroll
            for (int m = 0; m < 4; ++m) s_red[m][warp] = (double)vf[m];
        __syncthreads();
        if (threadIdx.x < 32) {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = lane < THREADS / 32 ? s_red[m][lane] : 0.0;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
#pragma unroll
                for (int m = 0; m < 4; ++m) v[m] += __shfl_down_sync(kFull, v[m], off);
            if (lane == 0) {
                const CheckArgs& ck = a.ck;
                const long long base = (long long)z * a.blocks_per_plane + bx;
                const long long plane_all = (long long)a.nz * a.blocks_per_plane;
#pragma unroll
                for (int m = 0; m < 4; ++m) *LBM_CK(ck.part + m * plane_all + base, ck.part, 4 * plane_all, 1, 6u) = v[m];
                // the last block of this plane to finish closes the plane
                __threadfence();
                const int ticket = atomicAdd(&ck.plane_cnt[z], 1);
                s_last = ticket == a.blocks_per_plane - 1;
            }
        }
        __syncthreads();
        if (s_last) close_plane<THREADS>(a, z);
    }
}

// Two fused steps (temporal blocking) in FP32.  A block owns FY rows of the
// full x extent (each thread 4 consecutive nodes, nq = nx / 4 threads per
// row) and marches through a chunk of planes.  Block row r = 0 .. FY + 1 is
// grid row y0 - 1 + r: rows 1 .. FY are the tile, rows 0 and FY + 1 the halo
// whose th and m_y the tile's second step pulls (populations 3 and 4).  The last tile of a
// cell whose ny is not a multiple of FY has fyb < FY rows; its halo is block
// row fyb + 1 and the rows after it idle.  Threads past (FY + 2) nq idle too
// (a batch launches every block with the same size).
// Iteration i computes step n + 1 at plane i - 2 for the tile rows (pulled
// from a ring of three shared planes, written to global memory) and step n
// at plane i for all rows (pulled from global memory, written to the ring).  Every node's arithmetic is the single step's
// (collide_node), so two fused steps equal two single steps bit for bit.
// Step n runs from frame rsrc to rdst, step n + 1 within rdst.
constexpr int F2_MAX_THREADS = 640;

// Kernel variants: rows of 128 nodes (tuned: 8-row tiles, 320 threads, two
// blocks per SM), 256 nodes (8-row tiles, 640 threads) and any multiple of 4
// (runtime row width); the launch bounds keep every variant at or below 96
// registers so that two 320-thread blocks fit an SM.
__host__ __device__ constexpr int f2_bound_threads(int nxc) { return nxc == 128 ? 320 : F2_MAX_THREADS; }
__host__ __device__ constexpr int f2_fixed_fy(int nxc) { return 8; }   // tile rows of the tuned variants
__host__ __device__ constexpr int f2_bound_blocks(int nxc) { return nxc == 128 ? 2 : 1; }

// A ring plane keeps, per field, only the rows the second step reads: th and
// m_y for block rows 0 .. FY + 1 (the y-neighbours of the tile rows), m_x and
// m_z for the FY tile rows.
__host__ __device__ constexpr int f2_slot_rows(int fy) { return 4 * fy + 4; }
__host__ __device__ constexpr size_t fused2_smem_bytes(int nx, int fy, int n_phases) {
    return sizeof(float) * 3 * (size_t)f2_slot_rows(fy) * nx + (sizeof(float4) + sizeof(float2)) * n_phases;
}

__device__ __forceinline__ float4 f4neg(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }
__device__ __forceinline__ float f4get(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// Step at 4 nodes of a row from the stored fields around them: th and m_x of
// the row (cT, cX) with the nodes left (lT, lX) and right (rT, rX) of it, th
// and m_y of the rows below (mT, mY) and above (pT, pY), th and m_z of the
// planes below (dT, dZ) and above (uT, uZ), faces already applied.
struct Quad4 {
    float4 o[kFields];                             // th, m_x, m_y, m_z of the 4 nodes
};
__device__ __forceinline__ Quad4 collide_quad(const float4& cT, const float4& cX, float lT, float lX, float rT,
                                              float rX, const float4& mT, const float4& mY, const float4& pT,
                                              const float4& pY, const float4& dT, const float4& dZ,
                                              const float4& uT, const float4& uZ, unsigned phw,
                                              const float4* s_sa, const float2* s_sc, float kT, float kJ) {
    Quad4 q;
    float* o = reinterpret_cast<float*>(q.o);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int ph = (phw >> (8 * k)) & 255u;
        const float2 sc = s_sc[ph];
        const float g0 = 0.25f * f4get(cT, k);
        const float g1 = k == 0 ? pull_p(lT, lX) : pull_p(f4get(cT, k - 1), f4get(cX, k - 1));
        const float g2 = k == 3 ? pull_m(rT, rX) : pull_m(f4get(cT, k + 1), f4get(cX, k + 1));
        const Collided c = collide_node(g0, g1, g2, pull_p(f4get(mT, k), f4get(mY, k)),
                                              pull_m(f4get(pT, k), f4get(pY, k)), pull_p(f4get(dT, k), f4get(dZ, k)),
                                              pull_m(f4get(uT, k), f4get(uZ, k)), s_sa[ph],
                                              make_float4(sc.x, sc.y, 0.f, 0.f), kT, kJ);
        o[k] = c.th;
        o[4 + k] = c.m[0];
        o[8 + k] = c.m[1];
        o[12 + k] = c.m[2];
    }
    return q;
}

// Loads the B tables into shared memory after the ring; returns the ring.
__device__ __forceinline__ float* fused2_tables(const StepArgs& a, int ring_floats, float4** s_sa,
                                                float2** s_sc) {
    extern __shared__ float4 smem4[];
    float* fn = reinterpret_cast<float*>(smem4);   // [3][f2_slot_rows][nx]
    // B per phase split into (xx, yy, zz, yz) and (xz, xy) tables: up to
    // 8 (16) distinct phases in a warp read one 128-byte wavefront
    *s_sa = reinterpret_cast<float4*>(fn + ring_floats);
    *s_sc = reinterpret_cast<float2*>(*s_sa + a.n_phases);
    for (int i = threadIdx.x; i < a.n_phases; i += blockDim.x) {
        (*s_sa)[i] = a.sb[2 * i];
        (*s_sc)[i] = make_float2(a.sb[2 * i + 1].x, a.sb[2 * i + 1].y);
    }
    return fn;
}

// One block of the two-step kernel: tile `by` of FY rows, chunk `bz` of
// zchunk planes.  NXC: compile-time row width (128, 256) or 0 (a.pitch).
// The caller has loaded the B tables (fused2_tables) but not yet synchronised.
template <bool PERIODIC, int NXC>
__device__ __forceinline__ void fused2_body(const StepArgs& a, float* fn, const float4* s_sa,
                                            const float2* s_sc, const int fy_arg, const int by, const int bz,
                                            const int zchunk, const int flip) {
    // the tuned row widths have a fixed tile height: every ring offset below
    // is then a compile-time constant
    const int FY = NXC ? f2_fixed_fy(NXC) : fy_arg;
    const int NXB = NXC ? NXC : a.pitch;           // nodes per row (= nx = pitch)
    const int nq = NXB >> 2;                       // threads per row
    // rows of whole warps: every branch on the row is warp-uniform, so a
    // warp whose row has no work skips the step (shuffles included)
    constexpr bool WR = NXC > 0 && NXC % 128 == 0;
    const int RS = f2_slot_rows(FY) * NXB;         // floats per ring plane
    // field offsets within a ring plane, relative to own = (r - 1) NXB + x of
    // block row r: th and m_y keep block rows 0 .. FY + 1, m_x and m_z rows
    // 1 .. FY
    const int QT = NXB, QY = (FY + 3) * NXB, QX = 2 * (FY + 2) * NXB, QZ = (3 * FY + 4) * NXB;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int r = tid / nq;                        // block row
    const int x = 4 * (tid - r * nq);              // first of this thread's 4 nodes
    const int ny = a.ny, nz = a.nz, pitch = a.pitch;
    const int y0 = by * FY;
    const int fyb = min(FY, ny - y0);              // tile rows of this block
    const bool live = r <= fyb + 1;
    int y = live ? y0 - 1 + r : 0;
    bool row_in = live;
    if (PERIODIC) y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    else row_in = live && y >= 0 && y < ny;
    const bool tile_row = r >= 1 && r <= fyb;
    const bool ylo = y == 0, yhi = y == ny - 1;
    const int xm = x == 0 ? NXB - 1 : x - 1;       // x - 1 of node x, wrapped
    const int xp = x + 4 == NXB ? 0 : x + 4;       // x + 1 of node x + 3, wrapped
    // x-neighbours come from the adjacent lane, except where that lane holds
    // another row or another warp holds the neighbour (a row of exactly one
    // warp wraps within the warp)
    const bool own_left = nq == 32 || !(lane == 0 || x == 0);
    const bool own_right = nq == 32 || !(lane == 31 || x + 4 == NXB);
    const long long P = a.pstride;
    const long long PL = (long long)ny * pitch;
    const long long yrow = (long long)y * pitch;
    // y-neighbour rows of the first step: the wrapped neighbour, or the own
    // row at an adiabatic face (Eq. 24, m_y with the other sign)
    const long long rym = ylo ? (PERIODIC ? yrow + (long long)(ny - 1) * pitch : yrow) : yrow - pitch;
    const long long ryp = yhi ? (PERIODIC ? yrow - (long long)(ny - 1) * pitch : yrow) : yrow + pitch;
    const float* __restrict__ src = reinterpret_cast<const float*>(a.src);
    float* __restrict__ dst = reinterpret_cast<float*>(a.dst);
    const int z0 = bz * zchunk;
    const int z1 = min(z0 + zchunk, nz);
    // chunks march alternately up and down, so that two neighbouring chunks
    // read the planes at their common boundary at about the same time; flip
    // reverses all of them (consecutive launches alternate, so a chunk starts
    // on the planes it wrote last)
    const bool up = ((bz & 1) == 0) == (flip == 0);
    const int dz = up ? 1 : -1;
    // frame constants of the two planes an iteration updates, computed one
    // iteration ahead by thread 0 into a double buffer: [t & 1][step n, n + 1]
    __shared__ PlaneK s_kc[2][2];
    auto plane_pair = [&](int t, PlaneK* out) {
        const int ii = up ? z0 - 1 + t : z1 - t;
        const int jj = ii - 2 * dz;
        out[0] = plane_consts(a.rsrc, a.rdst, min(max(ii, 0), nz - 1), nz, a.eps_hot, a.eps_cold);
        out[1] = plane_consts(a.rdst, a.rdst, min(max(jj, 0), nz - 1), nz, a.eps_hot, a.eps_cold);
    };
    if (tid == 0) plane_pair(0, s_kc[0]);
    __syncthreads();                               // the B tables and s_kc[0] are ready

    // L2 prefetch one plane ahead: lanes 0..4 of the block's last warp each
    // fetch, by one bulk prefetch, one field's rows that the tile's first
    // step reads there (th and m_y with the rows on either side, m_x and m_z
    // the block rows, clamped to the cell) or the phase bytes.  Plane i + 1
    // is read as the upper z-neighbour at the end of this iteration, after
    // the second step has given the prefetch time to land.  A bulk
    // prefetch takes its operands from uniform registers, so lanes with
    // different addresses are served one after another: one warp per block
    // keeps that loop short.
    const int pf_k = lane;                         // what this lane prefetches (< 5)
    const char* pf_base = nullptr;
    long long pf_plane = 4 * PL;                   // bytes per plane
    unsigned pf_bytes = 0u;
    {
        const int wide = (pf_k == 0 || pf_k == 2) ? 1 : 0;
        const int ya = max(y0 - 1 - wide, 0), yb = min(y0 + fyb + wide, ny - 1);
        const long long off = pf_k == 0 ? 0 : pf_k == 1 ? P : pf_k == 2 ? 2 * P : 3 * P;
        pf_base = reinterpret_cast<const char*>(src + off + (long long)ya * pitch);
        pf_bytes = yb >= ya ? 4u * (unsigned)((yb - ya + 1) * pitch) : 0u;
        if (pf_k == 4) {
            pf_base = reinterpret_cast<const char*>(a.phase + (long long)ya * pitch);
            pf_plane = PL;
            pf_bytes /= 4u;
        }
    }
    const bool pf_lane = (tid >> 5) == ((int)blockDim.x >> 5) - 1 && pf_k < 5 && pf_bytes > 0u &&
                         (pf_k != 4 || (pitch & 15) == 0);
    unsigned phA = 0u, phB = 0u;                   // phase words of planes i - 2dz and i - dz
    // ring slot of plane p: p mod 3.  si tracks plane i; planes j, j - 1 and
    // j + 1 then sit in slots si + 1, si, si + 2 (up) or si + 2, si + 1, si
    // (down), mod 3.
    int si = ((up ? z0 - 1 : z1) + 3) % 3;
    for (int t = 0; t < z1 - z0 + 3; ++t) {
        const int i = up ? z0 - 1 + t : z1 - t;    // step n at plane i
        const int j = i - 2 * dz;                  // step n + 1 at plane j
        const int s_inc = si == 2 ? 0 : si + 1, s_dec = si == 0 ? 2 : si - 1;
        const int sj = up ? s_inc : s_dec;
        const int sjm = up ? si : s_inc;           // plane j - 1
        const int sjp = up ? s_dec : si;           // plane j + 1
        const PlaneK kn = s_kc[t & 1][0], kn1 = s_kc[t & 1][1];
        if (tid == 0) plane_pair(t + 1, s_kc[(t + 1) & 1]);   // read after this iteration's barrier
        {
            const int ip = i + dz;
            if (pf_lane && ip >= max(z0 - 2, 0) && ip <= min(z1 + 1, nz - 1))
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(pf_base + ip * pf_plane),
                             "r"(pf_bytes) : "memory");
        }
        // ---- step n + 1 at plane j, tile rows ----
        const int own = (r - 1) * NXB + x;          // this thread's nodes in a ring plane
        const bool second = tile_row && j >= z0 && j < z1;
        if (!WR || second) {
            const float* fs = fn + sj * RS + own;
            const float* fb = fn + sjm * RS + own;
            const float* fa = fn + sjp * RS + own;
            float4 bT, bX, bmT, bmY, bpT, bpY, bdT, bdZ, buT, buZ;
            if (!WR && !second)
                bT = bX = bmT = bmY = bpT = bpY = bdT = bdZ = buT = buZ = make_float4(0.f, 0.f, 0.f, 0.f);
            if (WR || second) {
                const float* rb = fn;
                const int RN = 3 * RS;
                auto rd4 = [&](const float* q) { return *reinterpret_cast<const float4*>(LBM_CK(q, rb, RN, 4, 15u)); };
                bT = rd4(fs + QT);
                bX = rd4(fs + QX);
                if (PERIODIC || !ylo) {
                    bmT = rd4(fs + QT - NXB);
                    bmY = rd4(fs + QY - NXB);
                } else {
                    bmT = bT;
                    bmY = f4neg(rd4(fs + QY));
                }
                if (PERIODIC || !yhi) {
                    bpT = rd4(fs + QT + NXB);
                    bpY = rd4(fs + QY + NXB);
                } else {
                    bpT = bT;
                    bpY = f4neg(rd4(fs + QY));
                }
                if (j > 0) {
                    bdT = rd4(fb + QT);
                    bdZ = rd4(fb + QZ);
                } else {
                    bdT = f4neg(bT);
                    bdZ = rd4(fs + QZ);
                }
                if (j < nz - 1) {
                    buT = rd4(fa + QT);
                    buZ = rd4(fa + QZ);
                } else {
                    buT = f4neg(bT);
                    buZ = rd4(fs + QZ);
                }
            }
            // x-neighbours: from the next lane (every lane takes part), else
            // from the ring row
            float lT = __shfl_sync(kFull, bT.w, (lane + 31) & 31);
            float lX = __shfl_sync(kFull, bX.w, (lane + 31) & 31);
            float rT = __shfl_sync(kFull, bT.x, (lane + 1) & 31);
            float rX = __shfl_sync(kFull, bX.x, (lane + 1) & 31);
            if (WR || second) {
                if (!own_left) {
                    lT = *LBM_CK(fs + QT - x + xm, (const float*)fn, 3 * RS, 1, 15u);
                    lX = *LBM_CK(fs + QX - x + xm, (const float*)fn, 3 * RS, 1, 15u);
                }
                if (!own_right) {
                    rT = *LBM_CK(fs + QT - x + xp, (const float*)fn, 3 * RS, 1, 15u);
                    rX = *LBM_CK(fs + QX - x + xp, (const float*)fn, 3 * RS, 1, 15u);
                }
                if (!PERIODIC && x == 0) {                 // Eq. 24 at x = 0
                    lT = bT.x;
                    lX = -bX.x;
                }
                if (!PERIODIC && x + 4 == NXB) {           // and at x = nx - 1
                    rT = bT.w;
                    rX = -bX.w;
                }
                const Quad4 o = collide_quad(bT, bX, lT, lX, rT, rX, bmT, bmY, bpT, bpY, bdT, bdZ, buT, buZ, phA,
                                             s_sa, s_sc, kn1.kT, kn1.kJ);
                float* d = dst + (long long)j * PL + yrow + x;
#pragma unroll
                for (int f = 0; f < kFields; ++f)
                    *reinterpret_cast<float4*>(LBM_CK(d + f * P, dst, kFields * P, 4, 14u)) = o.o[f];
            }
        }
        // ---- loads of step n at plane i ----
        // issued after step n + 1: holding them in flight across that step
        // would need its registers too (the two-step kernel then spills); the
        // L2 prefetch of this plane two iterations ago keeps their latency short
        const bool first = i >= z0 - 1 && i <= z1 && i >= 0 && i < nz && row_in;
        float4 cT, cX, mT, mY, pT, pY, dT, dZ, uT, uZ;
        unsigned phC = 0u;
        if (first) {
            const float* s = src + (long long)i * PL;
            const float* sd = s + (i > 0 ? -PL : 0);          // the walls (Eq. 23) use the own node
            const float* su = s + (i < nz - 1 ? PL : 0);
            const int NP = kFields;
            cT = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + yrow + x, src, NP * P, 4, 11u)));
            cX = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + P + yrow + x, src, NP * P, 4, 11u)));
            mT = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + rym + x, src, NP * P, 4, 11u)));
            mY = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + 2 * P + rym + x, src, NP * P, 4, 11u)));
            pT = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + ryp + x, src, NP * P, 4, 11u)));
            pY = __ldg(reinterpret_cast<const float4*>(LBM_CK(s + 2 * P + ryp + x, src, NP * P, 4, 11u)));
            dT = __ldg(reinterpret_cast<const float4*>(LBM_CK(sd + yrow + x, src, NP * P, 4, 11u)));
            dZ = __ldg(reinterpret_cast<const float4*>(LBM_CK(sd + 3 * P + yrow + x, src, NP * P, 4, 11u)));
            uT = __ldg(reinterpret_cast<const float4*>(LBM_CK(su + yrow + x, src, NP * P, 4, 11u)));
            uZ = __ldg(reinterpret_cast<const float4*>(LBM_CK(su + 3 * P + yrow + x, src, NP * P, 4, 11u)));
            phC = __ldg(reinterpret_cast<const unsigned*>(
                LBM_CK(a.phase + (long long)i * PL + yrow + x, a.phase, P, 4, 12u)));
        } else if (!WR) {
            cT = cX = mT = mY = pT = pY = dT = dZ = uT = uZ = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // ---- step n at plane i into the ring ----
        if (!WR || first) {
            if (i == 0) dT = f4neg(dT);
            if (i == nz - 1) uT = f4neg(uT);
            if (!PERIODIC && ylo) mY = f4neg(mY);
            if (!PERIODIC && yhi) pY = f4neg(pY);
            float lT = __shfl_sync(kFull, cT.w, (lane + 31) & 31);
            float lX = __shfl_sync(kFull, cX.w, (lane + 31) & 31);
            float rT = __shfl_sync(kFull, cT.x, (lane + 1) & 31);
            float rX = __shfl_sync(kFull, cX.x, (lane + 1) & 31);
            if (WR || first) {
                const float* s = src + (long long)i * PL;
                if (!own_left) {
                    lT = __ldg(LBM_CK(s + yrow + xm, src, kFields * P, 1, 13u));
                    lX = __ldg(LBM_CK(s + P + yrow + xm, src, kFields * P, 1, 13u));
                }
                if (!own_right) {
                    rT = __ldg(LBM_CK(s + yrow + xp, src, kFields * P, 1, 13u));
                    rX = __ldg(LBM_CK(s + P + yrow + xp, src, kFields * P, 1, 13u));
                }
                if (!PERIODIC && x == 0) {
                    lT = cT.x;
                    lX = -cX.x;
                }
                if (!PERIODIC && x + 4 == NXB) {
                    rT = cT.w;
                    rX = -cX.w;
                }
                const Quad4 o = collide_quad(cT, cX, lT, lX, rT, rX, mT, mY, pT, pY, dT, dZ, uT, uZ, phC, s_sa,
                                             s_sc, kn.kT, kn.kJ);
                float* w = fn + si * RS + own;       // halo rows keep th and m_y only
                const int RN = 3 * RS;
                *reinterpret_cast<float4*>(LBM_CK(w + QT, fn, RN, 4, 16u)) = o.o[0];
                *reinterpret_cast<float4*>(LBM_CK(w + QY, fn, RN, 4, 16u)) = o.o[2];
                if (tile_row) {
                    *reinterpret_cast<float4*>(LBM_CK(w + QX, fn, RN, 4, 16u)) = o.o[1];
                    *reinterpret_cast<float4*>(LBM_CK(w + QZ, fn, RN, 4, 16u)) = o.o[3];
                }
            }
        }
        phA = phB;
        phB = phC;
        si = up ? s_inc : s_dec;
        __syncthreads();
    }
}

template <bool PERIODIC, int NXC>
__global__ void __launch_bounds__(f2_bound_threads(NXC), f2_bound_blocks(NXC))
    fused2_kernel(const StepArgs a, int fy, int zchunk, int flip) {
    const int NXB = NXC ? NXC : a.pitch;
    float4* s_sa;
    float2* s_sc;
    float* fn = fused2_tables(a, 3 * f2_slot_rows(fy) * NXB, &s_sa, &s_sc);
    fused2_body<PERIODIC, NXC>(a, fn, s_sa, s_sc, fy, blockIdx.x, blockIdx.y, zchunk, flip);
}

// Launch plan of the two-step kernel for a canonical nx x ny x nz cell:
// the kernel variant (nxc: 128, 256 or 0 for the runtime row width), tile
// height fy, block size, z chunk and grid.  The score estimates the useful
// fraction of the work: rows computed once per tile (fy of fy + 2 for the
// first step), planes computed once per chunk (zc of zc + 2), the fill of the
// last wave of blocks and the warps resident per SM (two blocks of 320
// threads measured best on rows of 128; one block per SM loses ~15 %).
struct F2Plan {
    bool ok;
    int nxc, fy, threads, zchunk, bxy, nzc;
    double score;
};

// force: take the best valid plan even for a cell too small to profit (the
// fused kernel on every shape, for tests and for choosing the layout).
template <typename Occ>
F2Plan f2_plan(int nx, int ny, int nz, int n_phases, int n_sm, int smem_max, bool force, Occ blocks_per_sm) {
    F2Plan best{};
    best.ok = false;
    best.score = -1.0;
    if (nx % 4 != 0 || nx < 4 || ny < 1 || nz < 1) return best;
    const int nq = nx / 4;
    const int nxc = nx == 128 ? 128 : (nx == 256 ? 256 : 0);
    const int fy_lo = nxc ? f2_fixed_fy(nxc) : 1;
    const int fy_hi = nxc ? f2_fixed_fy(nxc) : F2_MAX_THREADS / nq - 2;
    for (int fy = fy_lo; fy <= fy_hi; ++fy) {
        const int threads = (fy + 2) * nq;
        if (threads > f2_bound_threads(nxc)) break;
        if (threads < 128 && !force) continue;     // at least four warps per block
        const size_t smem = fused2_smem_bytes(nx, fy, n_phases);
        if (smem > (size_t)smem_max) break;
        const int nb = blocks_per_sm(nxc, threads, (size_t)smem);
        if (nb < 1) continue;
        const int bxy = (ny + fy - 1) / fy;
        const double rows = (double)ny / (double)(bxy * (fy + 2));
        const double occ = std::min(1.0, nb * threads / 640.0) * (nb >= 2 ? 1.0 : 0.85);
        const long long slots = (long long)nb * n_sm;
        for (int nzc = 1; nzc <= nz; ++nzc) {
            const int zc = (nz + nzc - 1) / nzc;
            if (nzc > 1 && zc < 4) break;
            const int nchunks = (nz + zc - 1) / zc;
            if (nchunks != nzc) continue;
            const long long blocks = (long long)bxy * nchunks;
            // a cell too small to give every SM a block runs single steps:
            // the two-step kernel's serial march through the planes would
            // only add latency there
            if (blocks < n_sm && !force) continue;
            const double fill = (double)blocks / (double)(((blocks + slots - 1) / slots) * slots);
            const double score = fill * zc / (zc + 2.0) * rows * occ;
            if (score > best.score + 1e-9) {
                best.ok = true;
                best.score = score;
                best.nxc = nxc;
                best.fy = fy;
                best.threads = threads;
                best.zchunk = zc;
                best.bxy = bxy;
                best.nzc = nchunks;
            }
        }
    }
    return best;
}

// The single-solve step: blockIdx.x is the block within the plane,
// blockIdx.y the plane, counted from the top when zrev is set: consecutive
// steps alternate, so that a step starts on the planes the previous one
// wrote last (still in L2).
template <int FMT, bool PERIODIC, bool CHECK, bool RAGGED>
__global__ void __launch_bounds__(kThreads, (CHECK && FMT != 0) ? 2 : 4) step_kernel(const StepArgs a) {
    const int z = a.zrev ? a.nz - 1 - (int)blockIdx.y : (int)blockIdx.y;
    step_body<FMT, PERIODIC, CHECK, RAGGED, kThreads>(a, blockIdx.x, z, a.rseed);
}

static __global__ void add_iters_kernel(Ctl* c, long long n) { c->iter += n; }

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
static __global__ void permute_phase_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, Layout L) {
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
// Value -> storage element (round to nearest; used only for the initial state).
template <int FMT> __device__ __forceinline__ typename Pol<FMT>::T to_store(float v);
template <> __device__ __forceinline__ float to_store<0>(float v) { return v; }
template <> __device__ __forceinline__ uint16_t to_store<1>(float v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ uint16_t to_store<2>(float v) {
    return __half_as_ushort(__float2half_rn(v));
}

// plane_th[z] = T0(z) - R(z) and plane_ts[z] = T0(z) - T_ref for the linear
// start (host FP64, rounded once); a caller field t_init replaces T0.
template <int FMT>
__global__ void init_kernel(void* __restrict__ fv, float* __restrict__ tsnap, long long P, Layout L,
                            const float* __restrict__ ref, const float* __restrict__ plane_th,
                            const float* __restrict__ plane_ts, float t_ref,
                            const float* __restrict__ t_init) {
    using T = typename Pol<FMT>::T;
    T* f = reinterpret_cast<T*>(fv);
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
                const float T0 = t_init[orig_index(L, xc, yc, zc)];
                th = T0 - ref[zc];
                ts = T0 - t_ref;
            } else {
                th = plane_th[zc];
                ts = plane_ts[zc];
            }
        }
        tsnap[i] = ts;
        f[i] = to_store<FMT>(th);                  // equilibrium: jhat = 0
        for (int q = 1; q < kFields; ++q) f[q * P + i] = to_store<FMT>(0.f);
    }
}

// T = sum_i f_i (Eq. 14) of the current state, written in the original order:
// the stored th plus the plane's reference.
template <int FMT>
__global__ void temperature_kernel(const void* __restrict__ fv, long long P, Layout L,
                                   const float* __restrict__ ref, float* __restrict__ T) {
    using S = Pol<FMT>;
    const typename S::T* f = reinterpret_cast<const typename S::T*>(fv);
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
        T[i] = S::scalar(f + k) + ref[zc];
    }
}

}  // namespace lbm
