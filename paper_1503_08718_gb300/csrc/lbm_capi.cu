// C ABI of the GB300 lattice Boltzmann solver (declared in include/lbm.h).
//
// Host responsibilities: validation, the FP64 material-to-lattice step
// (Eq. 12-13: tau = I/2 + s lambda / eps, S_b = tau^-1 per phase), laying the
// cell out with the Dirichlet axis slowest, device memory, and the CUDA graph
// that runs whole check intervals under a device-side while condition.  All
// per-voxel work runs in the kernels of lbm_kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_kernels.cuh"

using lbm::Ctl;
using lbm::Layout;

struct lbm_ctx {
    int n[3] = {0, 0, 0};
    int device = 0;
    int n_sm = 152;                        // multiprocessors of the device
    int l2_bytes = 0;                      // L2 cache of the device
    bool fuse_ok = false;                  // the two-step kernels got their shared memory
    int f2_smem_max = 0;                   // dynamic shared memory they may use (bytes)
    int pair_flip = 0;                     // chunk direction of the next lbm_advance pair
    mutable int step_flip = 0;             // plane order of the next single-step launch
    char* ws = nullptr;                    // caller's device workspace (nullptr: own allocations)
    size_t ws_bytes = 0;
    size_t ws_static = 0;                  // end of the part carved at creation
    double2* d_vox_anchor = nullptr;       // voxeliser scratch inside the workspace
    unsigned long long* d_vox_hist = nullptr;
    cudaStream_t own_stream = nullptr;     // context stream (non-blocking)
    cudaStream_t cap_stream = nullptr;     // private stream used only for graph capture
    bool poisoned = false;
    std::string err;

    // geometry and material (original order)
    uint8_t* d_phase = nullptr;            // nx*ny*nz
    int n_phases = 0;
    bool have_geometry = false;
    std::vector<double> lambda;            // n_phases*6
    bool have_tensors = false;

    // solve state
    bool started = false;
    int axis = 2, lateral = 0;
    lbm_solve_opts opts{};
    cudaStream_t stream = nullptr;         // stream used by the current solve
    Layout L{};
    char* d_f[2] = {nullptr, nullptr};     // distributions (4 or 2 bytes per value)
    size_t cap_f[2] = {0, 0};              // capacity of the f buffers (bytes)
    int fmt = 0;                           // lbm_storage of the current solve
    int cur = 0;                           // buffer holding the current state
    uint8_t* d_phase_c = nullptr;          // canonical padded phase map
    size_t cap_phase_c = 0;
    float* d_tsnap = nullptr;              // T - T_ref at the previous check (canonical)
    size_t cap_tsnap = 0;
    float* d_ref = nullptr;                // frames R_a, R_b, R_c [NZ each], then the
    size_t cap_ref = 0;                    // init tables T0 - R and T0 - T_ref [NZ each]
    double quantum = 0.0;                  // grid of the reference values
    float4* d_sb = nullptr;                // 2 float4 per phase
    int cap_sb = 0;
    double* d_part = nullptr;
    size_t cap_part = 0;
    double* d_Q = nullptr;                 // [NZ] plane flux, then [2][NZ] plane |dT|, |T|
    int cap_Q = 0;
    int* d_plane_cnt = nullptr;            // closing tickets per plane
    size_t cap_cnt = 0;
    float* d_T = nullptr;                  // nx*ny*nz staging (T output / t_init input)
    Ctl* d_ctl = nullptr;
    Ctl* h_ctl = nullptr;                  // pinned mirror
    double* d_hist = nullptr;              // per-check history ring [kHistCap][4]
    double s = 0.0;
    double t_ref = 0.0;
    int blocks_per_plane = 0;
    long long pstride = 0;
    std::vector<double> Q_host;
    std::vector<float> h_ref;              // staging of the initial reference frames
    double k_eff = NAN;
    bool have_k = false;

    // graph of one check interval inside a while node, one per buffer parity
    lbm::F2Plan f2{};                      // two-step kernel plan of the current solve
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    std::vector<char> gsig[2];             // kernel arguments baked into each graph
    int g_interval = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

constexpr int kHistCap = 1 << 16;          // checks kept in the history ring

// NVTX range for the duration of a scope (visible to Nsight tools; the
// header-only NVTX library costs nothing when no tool is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

lbm_status fail(lbm_ctx* c, lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CUDA_TRY(c, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (c)->poisoned = true;                                                           \
            return fail((c), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OUT_OF_MEMORY        \
                                                             : LBM_ERR_CUDA,                \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,   \
                        __LINE__);                                                          \
        }                                                                                   \
    } while (0)

#define CHECK_CTX(c)                                                                        \
    do {                                                                                    \
        if (!(c)) return LBM_ERR_INVALID_ARG;                                               \
        if ((c)->poisoned) return fail((c), LBM_ERR_CUDA, "context poisoned by an earlier CUDA error"); \
        (c)->err.clear();                                                                   \
    } while (0)

void free_graphs(lbm_ctx* c) {
    for (int p = 0; p < 2; ++p) {
        if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
        c->gexec[p] = nullptr;
        c->gsig[p].clear();
    }
    c->g_interval = 0;
}

// Cholesky test of a symmetric 3x3 tensor (xx, yy, zz, yz, xz, xy).
bool spd6(const double* t) {
    const double a00 = t[0], a11 = t[1], a22 = t[2], a12 = t[3], a02 = t[4], a01 = t[5];
    if (!(a00 > 0.0)) return false;
    const double l00 = std::sqrt(a00);
    const double l10 = a01 / l00, l20 = a02 / l00;
    const double d1 = a11 - l10 * l10;
    if (!(d1 > 0.0)) return false;
    const double l11 = std::sqrt(d1);
    const double l21 = (a12 - l20 * l10) / l11;
    const double d2 = a22 - l20 * l20 - l21 * l21;
    return d2 > 0.0 && std::isfinite(d2);
}

// Inverse of a symmetric 3x3 matrix (row-major) by cofactors, in FP64.
void inv3(const double* m, double* r) {
    const double c00 = m[4] * m[8] - m[5] * m[7];
    const double c01 = m[5] * m[6] - m[3] * m[8];
    const double c02 = m[3] * m[7] - m[4] * m[6];
    const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    r[0] = c00 / det;
    r[1] = (m[2] * m[7] - m[1] * m[8]) / det;
    r[2] = (m[1] * m[5] - m[2] * m[4]) / det;
    r[3] = c01 / det;
    r[4] = (m[0] * m[8] - m[2] * m[6]) / det;
    r[5] = (m[2] * m[3] - m[0] * m[5]) / det;
    r[6] = c02 / det;
    r[7] = (m[1] * m[6] - m[0] * m[7]) / det;
    r[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

int grid_1d(long long total) {
    long long b = (total + 255) / 256;
    if (b > 152LL * 32) b = 152LL * 32;
    return (int)(b < 1 ? 1 : b);
}

// Frames of the per-plane reference: the state between calls is relative to
// R_a; the first step of a graph interval moves it to R_b, and the check
// that closes the interval rotates R_a <- R_b <- new plane means.
enum Frame { kAA = 0, kAB = 1, kBB = 2 };

// How a check step closes: which frames rotate, how many iterations it
// closes and whether it drives a graph's while condition.
struct Closing {
    unsigned rseed = 0;                    // launch salt of the stochastic rounding
    int rebase = 0;
    int steps = 1;
    cudaGraphConditionalHandle handle = 0;
    int use_handle = 0;
};

lbm::StepArgs step_args(const lbm_ctx* c, int src, Frame fr, const Closing& cl = Closing()) {
    lbm::StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.src = c->d_f[src];
    a.dst = c->d_f[src ^ 1];
    a.phase = c->d_phase_c;
    a.sb = c->d_sb;
    a.tsnap = c->d_tsnap;
    const int NZ = c->L.NZ;
    float* ra = c->d_ref;
    float* rb = c->d_ref + NZ;
    a.rsrc = fr == kBB ? rb : ra;
    a.rdst = fr == kAA ? ra : rb;
    a.pstride = c->pstride;
    a.nx = c->L.NX;
    a.ny = c->L.NY;
    a.nz = NZ;
    a.pitch = c->L.pitch;
    a.n_phases = c->n_phases;
    a.quads_per_plane = (c->L.pitch / (c->fmt == LBM_STORE_F32 ? 4 : 8)) * c->L.NY;
    a.blocks_per_plane = c->blocks_per_plane;
    const double eps = 0.25;
    a.eps_hot = (float)(eps * c->opts.t_hot);
    a.eps_cold = (float)(eps * c->opts.t_cold);
    a.t_ref = c->t_ref;
    a.rseed = cl.rseed;
    lbm::CheckArgs& k = a.ck;
    k.part = c->d_part;
    k.Q = c->d_Q;
    k.plane = c->d_Q + NZ;
    k.plane_cnt = c->d_plane_cnt;
    k.ctl = c->d_ctl;
    k.ra = ra;
    k.rb = rb;
    k.rc = c->d_ref + 2 * NZ;
    k.rebase = cl.rebase;
    k.steps = cl.steps;
    k.stall_checks = c->opts.stall_checks;
    k.interval = c->opts.check_every;
    k.max_iters = c->opts.max_iters;
    k.tol = c->opts.tol;
    k.keff_scale = (double)NZ /
                   (c->s * (c->opts.t_hot - c->opts.t_cold) * (double)c->L.NX * (double)c->L.NY);
    k.inv_area = 1.0 / ((double)c->L.NX * (double)c->L.NY);
    k.quantum = c->quantum;
    k.inv_quantum = 1.0 / c->quantum;
    k.handle = cl.handle;
    k.use_handle = cl.use_handle;
    k.hist = c->d_hist;
    k.hist_cap = kHistCap;
    return a;
}

template <int FMT, bool RAGGED>
void launch_fmt(const lbm::StepArgs& a, bool periodic, bool check, dim3 grid, size_t smem,
                cudaStream_t st) {
    if (periodic) {
        if (check) lbm::step_kernel<FMT, true, true, RAGGED><<<grid, lbm::kThreads, smem, st>>>(a);
        else lbm::step_kernel<FMT, true, false, RAGGED><<<grid, lbm::kThreads, smem, st>>>(a);
    } else {
        if (check) lbm::step_kernel<FMT, false, true, RAGGED><<<grid, lbm::kThreads, smem, st>>>(a);
        else lbm::step_kernel<FMT, false, false, RAGGED><<<grid, lbm::kThreads, smem, st>>>(a);
    }
}

template <int FMT>
void launch_fmt(const lbm::StepArgs& a, bool periodic, bool check, bool ragged, dim3 grid,
                size_t smem, cudaStream_t st) {
    if (ragged) launch_fmt<FMT, true>(a, periodic, check, grid, smem, st);
    else launch_fmt<FMT, false>(a, periodic, check, grid, smem, st);
}

cudaError_t launch_step(const lbm_ctx* c, int src, bool check, Frame fr, cudaStream_t st,
                        const Closing& cl = Closing()) {
    lbm::StepArgs a = step_args(c, src, fr, cl);
    a.zrev = c->step_flip;                  // alternate launches reverse the plane order
    c->step_flip ^= 1;
    const dim3 grid(c->blocks_per_plane, c->L.NZ);
    const size_t smem = sizeof(float4) * 2 * c->n_phases;
    const bool periodic = c->lateral == LBM_LATERAL_PERIODIC;
    const bool ragged = c->L.NX != c->L.pitch;
    if (c->fmt == LBM_STORE_BF16) launch_fmt<1>(a, periodic, check, ragged, grid, smem, st);
    else if (c->fmt == LBM_STORE_F16) launch_fmt<2>(a, periodic, check, ragged, grid, smem, st);
    else launch_fmt<0>(a, periodic, check, ragged, grid, smem, st);
    return cudaGetLastError();
}

// Two plain FP32 steps in one launch (temporal blocking), when the layout
// allows it: rows of a multiple of 4 nodes (no padding).  The plan picks the
// tile height and the z chunk for the cell.
template <bool PER, int NXC>
const void* f2_kernel_ptr() {
    return reinterpret_cast<const void*>(lbm::fused2_kernel<PER, NXC>);
}

const void* f2_kernel(bool periodic, int nxc) {
    if (nxc == 128) return periodic ? f2_kernel_ptr<true, 128>() : f2_kernel_ptr<false, 128>();
    if (nxc == 256) return periodic ? f2_kernel_ptr<true, 256>() : f2_kernel_ptr<false, 256>();
    return periodic ? f2_kernel_ptr<true, 0>() : f2_kernel_ptr<false, 0>();
}

// Unless forced, the runtime-width variant is used only where the FP32 state
// (both buffers) exceeds twice the L2: below that, single steps run from L2
// at least as fast (measured on cubes of 64 to 176 nodes: single steps
// 82-204 GLUPS against 56-193 for the runtime-width two-step kernel; the
// tuned 128-node rows gain already at 128^3: 228 against 204).
lbm::F2Plan f2_plan_for(const lbm_ctx* c, int nx, int ny, int nz, int n_phases, bool periodic, bool force) {
    if (!c->fuse_ok) return lbm::F2Plan{};
    const bool tuned = nx == 128 || nx == 256;
    const double state = 2.0 * lbm::kFields * sizeof(float) * (double)nx * ny * nz;
    if (!force && !tuned && c->l2_bytes > 0 && state < 2.0 * c->l2_bytes) return lbm::F2Plan{};
    return lbm::f2_plan(nx, ny, nz, n_phases, c->n_sm, c->f2_smem_max, force,
                        [&](int nxc, int threads, size_t smem) {
                            int nb = 0;
                            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f2_kernel(periodic, nxc), threads,
                                                                              smem) != cudaSuccess) {
                                cudaGetLastError();
                                return 0;
                            }
                            return nb;
                        });
}

bool fusable(const lbm_ctx* c) {
    return c->opts.fuse && c->fmt == LBM_STORE_F32 && c->f2.ok;
}

// flip: 1 reverses every chunk's marching direction; alternate launches
// flip, so that each chunk starts on the planes it wrote last (still in L2).
cudaError_t launch_pair(const lbm_ctx* c, int src, Frame fr, int flip, cudaStream_t st) {
    const lbm::StepArgs a = step_args(c, src, fr);
    const lbm::F2Plan& p = c->f2;
    const dim3 grid(p.bxy, p.nzc);
    const size_t smem = lbm::fused2_smem_bytes(c->L.NX, p.fy, c->n_phases);
    const bool per = c->lateral == LBM_LATERAL_PERIODIC;
    if (p.nxc == 128) {
        if (per) lbm::fused2_kernel<true, 128><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
        else lbm::fused2_kernel<false, 128><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
    } else if (p.nxc == 256) {
        if (per) lbm::fused2_kernel<true, 256><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
        else lbm::fused2_kernel<false, 256><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
    } else {
        if (per) lbm::fused2_kernel<true, 0><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
        else lbm::fused2_kernel<false, 0><<<grid, p.threads, smem, st>>>(a, p.fy, p.zchunk, flip);
    }
    return cudaGetLastError();
}

// The launches of one check interval of K steps: a single step moving the
// state to frame R_b, plain steps (fused in an even number of pairs, so
// the interval ends in the buffer it started from), and the check step.
struct Plan {
    int pairs, singles;                  // plain steps after the first one
};

Plan interval_plan(const lbm_ctx* c) {
    const int R = c->opts.check_every - 2;
    Plan p;
    p.pairs = fusable(c) ? 2 * (R / 4) : 0;
    p.singles = R - 2 * p.pairs;
    return p;
}

// The closing of a graph or host-loop interval: the first step moved the
// state to frame R_b, and the check closes K iterations.
Closing interval_closing(const lbm_ctx* c) {
    Closing cl;
    cl.rebase = 1;
    cl.steps = c->opts.check_every;
    return cl;
}

// ---- workspace layout (lbm_create_with_workspace) ----
// Every device buffer of such a context is carved, 256-byte aligned and in a
// fixed order, from the caller's block: the creation-time part first, then,
// at each lbm_start, the buffers of that solve.  lbm_workspace_bytes adds
// up the same sizes.
constexpr size_t kWsAlign = 256;
constexpr int kWsYarns = 4096;             // voxeliser scratch for up to this many yarns
size_t ws_round(size_t x) { return (x + kWsAlign - 1) & ~(kWsAlign - 1); }

size_t ws_static_bytes(long long N) {
    return ws_round((size_t)N) + ws_round(sizeof(float) * (size_t)N) + ws_round(sizeof(Ctl)) +
           ws_round(sizeof(double) * 4 * kHistCap) + ws_round(sizeof(double2) * kWsYarns) +
           ws_round(sizeof(unsigned long long) * (kWsYarns + 1));
}

// the buffers lbm_start carves for a canonical NX x NY x NZ solve
size_t ws_solve_bytes(int NX, int NY, int NZ, int storage) {
    const int V = storage == LBM_STORE_F32 ? 4 : 8;
    const size_t esize = storage == LBM_STORE_F32 ? 4 : 2;
    const size_t pitch = (size_t)((NX + V - 1) / V * V);
    const size_t cells = pitch * NY * NZ;
    const size_t bpp = ((pitch / V) * NY + lbm::kThreads - 1) / lbm::kThreads;
    return 2 * ws_round(lbm::kFields * cells * esize) + ws_round(cells) + ws_round(sizeof(float) * cells) +
           ws_round(sizeof(float) * 5 * NZ) + ws_round(sizeof(int) * NZ) + ws_round(sizeof(float4) * 2 * 255) +
           ws_round(sizeof(double) * 4 * NZ * bpp) + ws_round(sizeof(double) * 3 * NZ);
}

template <typename T>
lbm_status ensure(lbm_ctx* c, T** p, size_t count, size_t* cap) {
    if (*p && *cap >= count) return LBM_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void**)p, sizeof(T) * count);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, LBM_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s",
                    sizeof(T) * count, cudaGetErrorString(e));
    }
    *cap = count;
    return LBM_OK;
}

// A solve's buffer: the context's own allocation, or the next piece of the
// caller's workspace (*cursor advances; a solve that does not fit fails).
template <typename T>
lbm_status solve_buf(lbm_ctx* c, size_t* cursor, T** p, size_t count, size_t* cap) {
    if (!c->ws) return ensure(c, p, count, cap);
    const size_t off = ws_round(*cursor);
    if (off + sizeof(T) * count > c->ws_bytes)
        return fail(c, LBM_ERR_OUT_OF_MEMORY,
                    "the workspace (%zu bytes) is too small for this solve; lbm_workspace_bytes gives "
                    "the size for this cell and storage", c->ws_bytes);
    *p = reinterpret_cast<T*>(c->ws + off);
    *cap = count;
    *cursor = off + sizeof(T) * count;
    return LBM_OK;
}

void fill_info(const lbm_ctx* c, lbm_solve_info* info, double ms) {
    if (!info) return;
    info->iters = c->h_ctl->iter;
    info->k_eff = c->h_ctl->k_eff;
    info->residual_T = c->h_ctl->r_t;
    info->residual_Q = c->h_ctl->r_q;
    info->elapsed_ms = ms;
    info->lattice_scale = c->s;
    info->status = c->h_ctl->status;
    info->checks = (int32_t)c->h_ctl->checks;
}

// The bounds-check word of this translation unit's kernels (bounds-checked
// builds only): a recorded code fails the call with LBM_ERR_INTERNAL.
lbm_status debug_word(lbm_ctx* c) {
#ifdef LBM_DEBUG
    unsigned code = 0;
    CUDA_TRY(c, cudaMemcpyFromSymbol(&code, lbm::g_lbm_debug, sizeof code));
    if (code) return fail(c, LBM_ERR_INTERNAL, "bounds check %u failed in a step kernel", code);
#else
    (void)c;
#endif
    return LBM_OK;
}

lbm_status read_ctl(lbm_ctx* c, cudaStream_t st) {
    CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaMemcpyAsync(c->Q_host.data(), c->d_Q, sizeof(double) * c->L.NZ,
                                cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    const lbm_status dbg = debug_word(c);
    if (dbg != LBM_OK) return dbg;
    c->k_eff = c->h_ctl->k_eff;
    c->have_k = c->h_ctl->checks > 0;
    return LBM_OK;
}

// Everything a check-interval graph bakes in: the kernel arguments of both
// buffer parities, the closing arguments, the lateral type and the storage.
std::vector<char> graph_signature(const lbm_ctx* c, int parity) {
    const lbm::StepArgs a = step_args(c, parity, kAB, interval_closing(c));
    std::vector<char> sig(sizeof a + 3 * sizeof(int));
    std::memcpy(sig.data(), &a, sizeof a);
    const int extra[3] = {c->lateral, c->opts.check_every,
                          (c->fmt * 2 + (fusable(c) ? 1 : 0)) | (c->f2.fy << 4) | (c->f2.zchunk << 12)};
    std::memcpy(sig.data() + sizeof a, extra, sizeof extra);
    return sig;
}

// Builds the executable graph: while (cond) { K-1 steps; check step }; the
// check step's closing block sets the condition.
lbm_status build_graph(lbm_ctx* c, int parity) {
    const int K = c->opts.check_every;
    cudaGraph_t g = nullptr;
    CUDA_TRY(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        c->poisoned = true;
        return fail(c, LBM_ERR_CUDA, "cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
    }
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        c->poisoned = true;
        return fail(c, LBM_ERR_CUDA, "cudaGraphAddNode(conditional): %s", cudaGetErrorString(e));
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        int src = parity;
        Closing cl = interval_closing(c);
        cl.handle = h;
        cl.use_handle = 1;
        const Plan pl = interval_plan(c);
        int k = 0;
        cl.rseed = (unsigned)k++;
        e = launch_step(c, src, false, kAB, c->cap_stream, cl);
        src ^= 1;
        for (int i = 0; i < pl.pairs && e == cudaSuccess; ++i, k += 2) {
            e = launch_pair(c, src, kBB, i & 1, c->cap_stream);
            src ^= 1;
        }
        for (int i = 0; i < pl.singles && e == cudaSuccess; ++i) {
            cl.rseed = (unsigned)k++;
            e = launch_step(c, src, false, kBB, c->cap_stream, cl);
            src ^= 1;
        }
        if (e == cudaSuccess) {
            cl.rseed = (unsigned)k;
            e = launch_step(c, src, true, kBB, c->cap_stream, cl);
            src ^= 1;
        }
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &captured);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec[parity] = nullptr;
        c->poisoned = true;
        return fail(c, LBM_ERR_CUDA, "building the check-interval graph failed: %s",
                    cudaGetErrorString(e));
    }
    c->g_interval = K;
    c->gsig[parity] = graph_signature(c, parity);
    return LBM_OK;
}

}  // namespace

extern "C" {

void lbm_default_opts(lbm_solve_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->t_hot = 1.0;
    o->t_cold = 0.0;
    o->tau_max = 1.5;
    o->lattice_scale = 0.0;
    o->tol = 1e-8;
    o->max_iters = 50000000LL;
    o->check_every = 100;
    o->stall_checks = 0;
    o->storage = LBM_STORE_F32;
    o->fuse = 1;
    o->t_init = nullptr;
    o->stream = nullptr;
}

namespace {

// Creation shared by lbm_create (ws == nullptr: own allocations) and
// lbm_create_with_workspace (every device buffer carved from ws).
lbm_status create_ctx(int nx, int ny, int nz, int cuda_device, char* ws, size_t ws_bytes, lbm_ctx** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2) return LBM_ERR_INVALID_ARG;
    const long long N = (long long)nx * ny * nz;
    if (N >= (1LL << 31)) return LBM_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
        cudaGetLastError();
        return LBM_ERR_INVALID_ARG;
    }
    lbm_ctx* c = new (std::nothrow) lbm_ctx();
    if (!c) return LBM_ERR_OUT_OF_MEMORY;
    c->n[0] = nx;
    c->n[1] = ny;
    c->n[2] = nz;
    c->device = cuda_device;
    lbm_default_opts(&c->opts);
    bool ok = cudaSetDevice(cuda_device) == cudaSuccess;
    if (ok && ws) {
        size_t off = 0;
        auto carve = [&](size_t bytes) {
            char* p = ws + off;
            off = ws_round(off + bytes);
            return p;
        };
        c->ws = ws;
        c->ws_bytes = ws_bytes;
        c->d_phase = reinterpret_cast<uint8_t*>(carve((size_t)N));
        c->d_T = reinterpret_cast<float*>(carve(sizeof(float) * (size_t)N));
        c->d_ctl = reinterpret_cast<Ctl*>(carve(sizeof(Ctl)));
        c->d_hist = reinterpret_cast<double*>(carve(sizeof(double) * 4 * kHistCap));
        c->d_vox_anchor = reinterpret_cast<double2*>(carve(sizeof(double2) * kWsYarns));
        c->d_vox_hist = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long) * (kWsYarns + 1)));
        c->ws_static = off;
    } else if (ok) {
        ok = cudaMalloc((void**)&c->d_phase, (size_t)N) == cudaSuccess &&
             cudaMalloc((void**)&c->d_T, sizeof(float) * (size_t)N) == cudaSuccess &&
             cudaMalloc((void**)&c->d_ctl, sizeof(Ctl)) == cudaSuccess &&
             cudaMalloc((void**)&c->d_hist, sizeof(double) * 4 * kHistCap) == cudaSuccess;
    }
    ok = ok && cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMallocHost((void**)&c->h_ctl, sizeof(Ctl)) == cudaSuccess &&
              cudaEventCreate(&c->ev0) == cudaSuccess && cudaEventCreate(&c->ev1) == cudaSuccess &&
              cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, cuda_device) == cudaSuccess &&
              cudaDeviceGetAttribute(&c->l2_bytes, cudaDevAttrL2CacheSize, cuda_device) == cudaSuccess;
    // the fused two-step kernels need more than the default 48 KB of shared
    // memory; without it every solve runs single steps
    if (ok) {
        int optin = 0;
        c->fuse_ok = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, cuda_device) ==
                     cudaSuccess;
        int most = optin;
        for (int per = 0; per < 2 && c->fuse_ok; ++per)
            for (int nxc : {128, 256, 0}) {
                const void* k = f2_kernel(per == 1, nxc);
                cudaFuncAttributes fa;
                if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) {
                    c->fuse_ok = false;
                    break;
                }
                const int dyn = optin - (int)fa.sharedSizeBytes;
                most = std::min(most, dyn);
                c->fuse_ok = c->fuse_ok && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                                dyn) == cudaSuccess;
            }
        c->f2_smem_max = c->fuse_ok ? most : 0;
        cudaGetLastError();
    }
    if (!ok) {
        cudaGetLastError();
        lbm_destroy(c);
        return LBM_ERR_OUT_OF_MEMORY;
    }
    std::memset(c->h_ctl, 0, sizeof(Ctl));
    *out = c;
    return LBM_OK;
}

}  // namespace

lbm_status lbm_create(int nx, int ny, int nz, int cuda_device, lbm_ctx** out) {
    return create_ctx(nx, ny, nz, cuda_device, nullptr, 0, out);
}

size_t lbm_workspace_bytes(int nx, int ny, int nz, int storage) {
    if (nx < 2 || ny < 2 || nz < 2 || (long long)nx * ny * nz >= (1LL << 31)) return 0;
    if (storage != LBM_STORE_F32 && storage != LBM_STORE_BF16 && storage != LBM_STORE_F16) return 0;
    const int n[3] = {nx, ny, nz};
    size_t most = 0;
    // any Dirichlet axis, either order of the two lateral axes
    for (int a = 0; a < 3; ++a)
        for (int o = 0; o < 2; ++o) {
            const int b = (a + 1 + o) % 3, d = (a + 2 - o) % 3;
            most = std::max(most, ws_solve_bytes(n[b], n[d], n[a], storage));
        }
    return ws_static_bytes((long long)nx * ny * nz) + most;
}

lbm_status lbm_create_with_workspace(int nx, int ny, int nz, int cuda_device, void* dev_ptr, size_t bytes,
                                     lbm_ctx** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & (kWsAlign - 1)) != 0) return LBM_ERR_INVALID_ARG;
    if (nx < 2 || ny < 2 || nz < 2 || (long long)nx * ny * nz >= (1LL << 31)) return LBM_ERR_INVALID_ARG;
    if (bytes < ws_static_bytes((long long)nx * ny * nz)) return LBM_ERR_INVALID_ARG;
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, dev_ptr) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
        pa.device != cuda_device) {
        cudaGetLastError();
        return LBM_ERR_INVALID_ARG;
    }
    return create_ctx(nx, ny, nz, cuda_device, static_cast<char*>(dev_ptr), bytes, out);
}

lbm_status lbm_set_geometry(lbm_ctx* c, const uint8_t* phase, int n_phases) {
    CHECK_CTX(c);
    if (!phase) return fail(c, LBM_ERR_INVALID_ARG, "phase is NULL");
    if (n_phases < 1 || n_phases > 255) return fail(c, LBM_ERR_INVALID_ARG, "n_phases must be in [1, 255]");
    const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    // largest id first (a branch-free scan the compiler vectorises), then the
    // first offending voxel only if there is one
    uint8_t top = 0;
    for (size_t i = 0; i < N; ++i) top = phase[i] > top ? phase[i] : top;
    if (top >= n_phases)
        for (size_t i = 0; i < N; ++i)
            if (phase[i] >= n_phases)
                return fail(c, LBM_ERR_INVALID_ARG, "phase id %d at voxel %zu is >= n_phases %d",
                            (int)phase[i], i, n_phases);
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaMemcpy(c->d_phase, phase, N, cudaMemcpyHostToDevice));
    if (c->have_tensors && (int)c->lambda.size() != 6 * n_phases) c->have_tensors = false;
    c->n_phases = n_phases;
    c->have_geometry = true;
    c->started = false;
    return LBM_OK;
}

lbm_status lbm_set_tensors(lbm_ctx* c, const double* lambda, int n_phases) {
    CHECK_CTX(c);
    if (!lambda) return fail(c, LBM_ERR_INVALID_ARG, "lambda is NULL");
    if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "set the geometry before the tensors");
    if (n_phases != c->n_phases)
        return fail(c, LBM_ERR_INVALID_ARG, "n_phases %d does not match the geometry's %d", n_phases,
                    c->n_phases);
    for (int p = 0; p < n_phases; ++p) {
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(lambda[6 * p + k]))
                return fail(c, LBM_ERR_INVALID_ARG, "tensor of phase %d is not finite", p);
        if (!spd6(lambda + 6 * p))
            return fail(c, LBM_ERR_INVALID_ARG, "tensor of phase %d is not positive definite", p);
    }
    c->lambda.assign(lambda, lambda + 6 * n_phases);
    c->have_tensors = true;
    c->started = false;
    return LBM_OK;
}

lbm_status lbm_start(lbm_ctx* c, lbm_axis axis, lbm_lateral lateral, const lbm_solve_opts* o) {
    CHECK_CTX(c);
    NvtxRange nvtx("lbm_start");
    if (!c->have_geometry || !c->have_tensors)
        return fail(c, LBM_ERR_STATE, "set geometry and tensors before starting a solve");
    if (axis < LBM_AXIS_X || axis > LBM_AXIS_Z) return fail(c, LBM_ERR_INVALID_ARG, "bad axis");
    if (lateral != LBM_LATERAL_PERIODIC && lateral != LBM_LATERAL_ADIABATIC)
        return fail(c, LBM_ERR_INVALID_ARG, "bad lateral type");
    lbm_solve_opts op;
    if (o) op = *o;
    else lbm_default_opts(&op);
    if (!(op.t_hot != op.t_cold) || !std::isfinite(op.t_hot) || !std::isfinite(op.t_cold))
        return fail(c, LBM_ERR_INVALID_ARG, "t_hot and t_cold must be finite and differ");
    if (op.check_every < 2 || (op.check_every & 1) || op.check_every > 4096)
        return fail(c, LBM_ERR_INVALID_ARG, "check_every must be even and in [2, 4096]");
    if (op.max_iters < 0) return fail(c, LBM_ERR_INVALID_ARG, "max_iters must be >= 0");
    if (op.storage != LBM_STORE_F32 && op.storage != LBM_STORE_BF16 && op.storage != LBM_STORE_F16)
        return fail(c, LBM_ERR_INVALID_ARG, "unsupported storage");
    if (!(op.lattice_scale > 0.0) && !(op.tau_max > 0.5))
        return fail(c, LBM_ERR_INVALID_ARG, "tau_max must exceed 1/2");
    CUDA_TRY(c, cudaSetDevice(c->device));

    // lattice scale and S_b = tau^-1 per phase (Eq. 12-13), FP64 on the host
    const double eps = 0.25;
    double s = op.lattice_scale;
    if (!(s > 0.0)) {
        double m = 0.0;
        for (int p = 0; p < c->n_phases; ++p)
            for (int k = 0; k < 3; ++k) m = std::fmax(m, c->lambda[6 * p + k]);
        s = eps * (op.tau_max - 0.5) / m;
    }
    // canonical layout: new axis i is old axis perm[i], Dirichlet axis last.
    // Either order of the two lateral axes is valid (the tensors are permuted
    // with the map); take the one whose rows the two-step kernel accepts.
    static const int perms[3][3] = {{1, 2, 0}, {2, 0, 1}, {0, 1, 2}};
    Layout L;
    for (int i = 0; i < 3; ++i) {
        L.n[i] = c->n[i];
        L.perm[i] = perms[axis][i];
    }
    // (the order depends on the geometry only, not on opts.fuse, so that a
    // solve with fused pairs and one without share the layout bit for bit)
    lbm::F2Plan f2{};
    if (op.storage == LBM_STORE_F32) {
        const bool per = lateral == LBM_LATERAL_PERIODIC;
        const lbm::F2Plan a0 = f2_plan_for(c, c->n[L.perm[0]], c->n[L.perm[1]], c->n[L.perm[2]], c->n_phases, per, true);
        const lbm::F2Plan a1 = f2_plan_for(c, c->n[L.perm[1]], c->n[L.perm[0]], c->n[L.perm[2]], c->n_phases, per, true);
        if (a1.ok && (!a0.ok || a1.score > a0.score * 1.001)) {
            const int t = L.perm[0];
            L.perm[0] = L.perm[1];
            L.perm[1] = t;
        }
        // fuse = 2 takes the two-step kernel even where it would not pay
        if (op.fuse)
            f2 = f2_plan_for(c, c->n[L.perm[0]], c->n[L.perm[1]], c->n[L.perm[2]], c->n_phases, per, op.fuse == 2);
    }
    L.NX = c->n[L.perm[0]];
    L.NY = c->n[L.perm[1]];
    L.NZ = c->n[L.perm[2]];
    const int V = op.storage == LBM_STORE_F32 ? 4 : 8;       // voxels per thread
    const size_t esize = op.storage == LBM_STORE_F32 ? 4 : 2;
    L.pitch = (L.NX + V - 1) / V * V;
    if (L.NZ > 65535)
        return fail(c, LBM_ERR_INVALID_ARG, "the temperature-difference axis may have at most 65535 nodes");
    std::vector<float4> sb(2 * (size_t)c->n_phases);
    for (int p = 0; p < c->n_phases; ++p) {
        const double* t = &c->lambda[6 * p];
        const double full[9] = {t[0], t[5], t[4], t[5], t[1], t[3], t[4], t[3], t[2]};
        double lam[9], tau[9], S[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) lam[3 * i + j] = full[3 * L.perm[i] + L.perm[j]];
        for (int k = 0; k < 9; ++k) tau[k] = s * lam[k] / eps;
        tau[0] += 0.5;
        tau[4] += 0.5;
        tau[8] += 0.5;
        inv3(tau, S);
        // the device's per-phase table: B = (I - S_b) / 2 for FP32, S_b for 16 bits
        lbm::phase_entry(S, &sb[2 * (size_t)p]);
    }

    // buffers
    const long long cells = (long long)L.pitch * L.NY * L.NZ;
    lbm_status st;
    size_t cur = c->ws_static;              // workspace cursor (unused without a workspace)
    if ((st = solve_buf(c, &cur, &c->d_f[0], (size_t)(lbm::kFields * cells) * esize, &c->cap_f[0])) != LBM_OK) return st;
    if ((st = solve_buf(c, &cur, &c->d_f[1], (size_t)(lbm::kFields * cells) * esize, &c->cap_f[1])) != LBM_OK) return st;
    if ((st = solve_buf(c, &cur, &c->d_phase_c, (size_t)cells, &c->cap_phase_c)) != LBM_OK) return st;
    if ((st = solve_buf(c, &cur, &c->d_tsnap, (size_t)cells, &c->cap_tsnap)) != LBM_OK) return st;
    if ((st = solve_buf(c, &cur, &c->d_ref, (size_t)5 * L.NZ, &c->cap_ref)) != LBM_OK) return st;
    if ((st = solve_buf(c, &cur, &c->d_plane_cnt, (size_t)L.NZ, &c->cap_cnt)) != LBM_OK) return st;
    size_t cap_sb = (size_t)c->cap_sb;
    if ((st = solve_buf(c, &cur, &c->d_sb, c->ws ? (size_t)2 * 255 : sb.size(), &cap_sb)) != LBM_OK) return st;
    c->cap_sb = (int)cap_sb;
    const int quads = (L.pitch / V) * L.NY;
    c->blocks_per_plane = (quads + lbm::kThreads - 1) / lbm::kThreads;
    if ((st = solve_buf(c, &cur, &c->d_part, (size_t)4 * L.NZ * c->blocks_per_plane, &c->cap_part)) != LBM_OK)
        return st;
    size_t capQ = (size_t)c->cap_Q;
    if ((st = solve_buf(c, &cur, &c->d_Q, (size_t)3 * L.NZ, &capQ)) != LBM_OK) return st;
    c->cap_Q = (int)capQ;
    c->Q_host.assign(L.NZ, 0.0);

    c->opts = op;
    c->f2 = f2;
    c->fmt = op.storage;
    c->axis = axis;
    c->lateral = lateral;
    c->L = L;
    c->s = s;
    c->t_ref = 0.5 * (op.t_hot + op.t_cold);
    c->pstride = cells;
    c->stream = op.stream ? (cudaStream_t)op.stream : c->own_stream;
    c->cur = 0;
    c->have_k = false;
    c->k_eff = NAN;

    cudaStream_t stm = c->stream;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_sb, sb.data(), sizeof(float4) * sb.size(),
                                cudaMemcpyHostToDevice, stm));
    lbm::permute_phase_kernel<<<grid_1d(cells), 256, 0, stm>>>(c->d_phase, c->d_phase_c, L);
    CUDA_TRY(c, cudaGetLastError());
    // initial reference frame: the plane means of the initial field on the
    // quantum grid 2^(e-20), 2^e >= max |T_wall|, so that w (R - R') is exact
    int e2 = 0;
    std::frexp(std::fmax(std::fmax(std::fabs(op.t_hot), std::fabs(op.t_cold)), 1.0), &e2);
    c->quantum = std::ldexp(1.0, e2 - 20);
    std::vector<double> mean(L.NZ, 0.0);
    const float* tinit = nullptr;
    if (op.t_init) {
        const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
        for (size_t i = 0; i < N; ++i) {
            int cc[3] = {(int)(i % c->n[0]), (int)((i / c->n[0]) % c->n[1]),
                         (int)(i / ((size_t)c->n[0] * c->n[1]))};
            mean[cc[L.perm[2]]] += op.t_init[i];
        }
        for (auto& m : mean) m /= (double)L.NX * (double)L.NY;
        CUDA_TRY(c, cudaMemcpyAsync(c->d_T, op.t_init, sizeof(float) * N, cudaMemcpyHostToDevice, stm));
        tinit = c->d_T;
    } else {
        for (int z = 0; z < L.NZ; ++z)
            mean[z] = op.t_hot + (op.t_cold - op.t_hot) * ((double)z + 0.5) / (double)L.NZ;
    }
    c->h_ref.assign(5 * (size_t)L.NZ, 0.f);
    for (int z = 0; z < L.NZ; ++z) {
        const double r = std::nearbyint(mean[z] / c->quantum) * c->quantum;
        const double T0 = op.t_hot + (op.t_cold - op.t_hot) * ((double)z + 0.5) / (double)L.NZ;
        c->h_ref[z] = (float)r;
        c->h_ref[L.NZ + z] = (float)r;
        c->h_ref[2 * L.NZ + z] = (float)r;
        c->h_ref[3 * L.NZ + z] = (float)(T0 - r);
        c->h_ref[4 * L.NZ + z] = (float)(T0 - c->t_ref);
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ref, c->h_ref.data(), sizeof(float) * 5 * L.NZ,
                                cudaMemcpyHostToDevice, stm));
    CUDA_TRY(c, cudaMemsetAsync(c->d_plane_cnt, 0, sizeof(int) * L.NZ, stm));
    {
        const float* th = c->d_ref + 3 * L.NZ;
        const float* ts = c->d_ref + 4 * L.NZ;
        const int g = grid_1d(cells);
        if (op.storage == LBM_STORE_BF16)
            lbm::init_kernel<1><<<g, 256, 0, stm>>>(c->d_f[0], c->d_tsnap, cells, L, c->d_ref, th, ts,
                                                   (float)c->t_ref, tinit);
        else if (op.storage == LBM_STORE_F16)
            lbm::init_kernel<2><<<g, 256, 0, stm>>>(c->d_f[0], c->d_tsnap, cells, L, c->d_ref, th, ts,
                                                   (float)c->t_ref, tinit);
        else
            lbm::init_kernel<0><<<g, 256, 0, stm>>>(c->d_f[0], c->d_tsnap, cells, L, c->d_ref, th, ts,
                                                   (float)c->t_ref, tinit);
    }
    CUDA_TRY(c, cudaGetLastError());
    Ctl h{};
    h.best_rt = INFINITY;
    h.k_eff = NAN;
    h.r_t = NAN;
    h.r_q = NAN;
    h.status = LBM_ERR_NOT_CONVERGED;
    *c->h_ctl = h;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ctl, c->h_ctl, sizeof(Ctl), cudaMemcpyHostToDevice, stm));
    CUDA_TRY(c, cudaStreamSynchronize(stm));
    c->started = true;
    return LBM_OK;
}

lbm_status lbm_advance(lbm_ctx* c, int64_t n_steps) {
    CHECK_CTX(c);
    NvtxRange nvtx("lbm_advance");
    if (!c->started) return fail(c, LBM_ERR_STATE, "call lbm_start first");
    if (n_steps < 0) return fail(c, LBM_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (n_steps == 0) return LBM_OK;
    CUDA_TRY(c, cudaSetDevice(c->device));
    int64_t k = 0;
    if (fusable(c)) {
        for (; k + 2 <= n_steps; k += 2) {
            CUDA_TRY(c, launch_pair(c, c->cur, kAA, c->pair_flip, c->stream));
            c->pair_flip ^= 1;
            c->cur ^= 1;
        }
    }
    for (; k < n_steps; ++k) {
        Closing cl;
        cl.rseed = 0x10000u + (unsigned)k;
        CUDA_TRY(c, launch_step(c, c->cur, false, kAA, c->stream, cl));
        c->cur ^= 1;
    }
    lbm::add_iters_kernel<<<1, 1, 0, c->stream>>>(c->d_ctl, (long long)n_steps);
    CUDA_TRY(c, cudaGetLastError());
    return LBM_OK;
}

lbm_status lbm_check(lbm_ctx* c, lbm_solve_info* info) {
    CHECK_CTX(c);
    NvtxRange nvtx("lbm_check");
    if (!c->started) return fail(c, LBM_ERR_STATE, "call lbm_start first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    Closing cl;
    cl.rseed = 0x5bd1e995u;
    CUDA_TRY(c, launch_step(c, c->cur, true, kAA, c->stream, cl));
    c->cur ^= 1;
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    lbm_status st = read_ctl(c, c->stream);
    if (st != LBM_OK) return st;
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    fill_info(c, info, ms);
    return LBM_OK;
}

lbm_status lbm_run(lbm_ctx* c, lbm_solve_info* info) {
    CHECK_CTX(c);
    NvtxRange nvtx("lbm_run");
    if (!c->started) return fail(c, LBM_ERR_STATE, "call lbm_start first");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const int K = c->opts.check_every;
    // the stop rule needs the current iteration count
    lbm_status st = read_ctl(c, c->stream);
    if (st != LBM_OK) return st;
    if (c->h_ctl->iter + K > c->opts.max_iters) {
        fill_info(c, info, 0.0);
        if (info) info->status = LBM_ERR_NOT_CONVERGED;
        return fail(c, LBM_ERR_NOT_CONVERGED, "max_iters leaves no whole check interval to run");
    }
    CUDA_TRY(c, cudaEventRecord(c->ev0, c->stream));
    if (c->opts.host_loop) {
        // the same interval, launched kernel by kernel; the stop flag is read
        // back after every interval
        do {
            const Plan pl = interval_plan(c);
            Closing cl = interval_closing(c);
            int k = 0;
            cl.rseed = (unsigned)k++;
            CUDA_TRY(c, launch_step(c, c->cur, false, kAB, c->stream, cl));
            c->cur ^= 1;
            for (int i = 0; i < pl.pairs; ++i, k += 2) {
                CUDA_TRY(c, launch_pair(c, c->cur, kBB, i & 1, c->stream));
                c->cur ^= 1;
            }
            for (int i = 0; i < pl.singles; ++i) {
                cl.rseed = (unsigned)k++;
                CUDA_TRY(c, launch_step(c, c->cur, false, kBB, c->stream, cl));
                c->cur ^= 1;
            }
            cl.rseed = (unsigned)k;
            CUDA_TRY(c, launch_step(c, c->cur, true, kBB, c->stream, cl));
            c->cur ^= 1;
            CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                        c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        } while (!c->h_ctl->done);
    } else {
        // reuse the graph of an earlier solve when nothing it bakes in changed
        if (!c->gexec[c->cur] || c->gsig[c->cur] != graph_signature(c, c->cur)) {
            if (c->gexec[c->cur]) cudaGraphExecDestroy(c->gexec[c->cur]);
            c->gexec[c->cur] = nullptr;
            if ((st = build_graph(c, c->cur)) != LBM_OK) return st;
        }
        CUDA_TRY(c, cudaGraphLaunch(c->gexec[c->cur], c->stream));
    }
    CUDA_TRY(c, cudaEventRecord(c->ev1, c->stream));
    if ((st = read_ctl(c, c->stream)) != LBM_OK) return st;
    // K is even, so the state is back in the buffer it started from
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    fill_info(c, info, ms);
    const int s = c->h_ctl->status;
    if (s == LBM_OK) return LBM_OK;
    if (s == LBM_ERR_DIVERGED) return fail(c, LBM_ERR_DIVERGED, "non-finite residual or flux");
    if (s == LBM_ERR_STALLED) return fail(c, LBM_ERR_STALLED, "residual stalled at %.3e", c->h_ctl->r_t);
    return fail(c, LBM_ERR_NOT_CONVERGED, "max_iters reached with R_T = %.3e", c->h_ctl->r_t);
}

lbm_status lbm_solve(lbm_ctx* c, lbm_axis axis, lbm_lateral lateral, const lbm_solve_opts* o,
                     lbm_solve_info* info) {
    lbm_status st = lbm_start(c, axis, lateral, o);
    if (st != LBM_OK) return st;
    return lbm_run(c, info);
}

lbm_status lbm_k_eff(const lbm_ctx* c, double* out) {
    if (!c || !out) return LBM_ERR_INVALID_ARG;
    if (c->poisoned) return LBM_ERR_CUDA;
    if (!c->have_k) return LBM_ERR_STATE;
    *out = c->k_eff;
    return LBM_OK;
}

lbm_status lbm_get_temperature(lbm_ctx* c, float* host_out) {
    CHECK_CTX(c);
    if (!host_out) return fail(c, LBM_ERR_INVALID_ARG, "host_out is NULL");
    if (!c->started) return fail(c, LBM_ERR_STATE, "no solve state");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const long long N = (long long)c->n[0] * c->n[1] * c->n[2];
    if (c->fmt == LBM_STORE_BF16)
        lbm::temperature_kernel<1><<<grid_1d(N), 256, 0, c->stream>>>(c->d_f[c->cur], c->pstride, c->L,
                                                                     c->d_ref, c->d_T);
    else if (c->fmt == LBM_STORE_F16)
        lbm::temperature_kernel<2><<<grid_1d(N), 256, 0, c->stream>>>(c->d_f[c->cur], c->pstride, c->L,
                                                                     c->d_ref, c->d_T);
    else
        lbm::temperature_kernel<0><<<grid_1d(N), 256, 0, c->stream>>>(c->d_f[c->cur], c->pstride, c->L,
                                                                     c->d_ref, c->d_T);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaMemcpyAsync(host_out, c->d_T, sizeof(float) * N, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

lbm_status lbm_get_plane_flux(const lbm_ctx* c, double* host_out, int n) {
    if (!c || !host_out) return LBM_ERR_INVALID_ARG;
    if (c->poisoned) return LBM_ERR_CUDA;
    if (!c->have_k) return LBM_ERR_STATE;
    if (n != c->L.NZ) return LBM_ERR_INVALID_ARG;
    std::memcpy(host_out, c->Q_host.data(), sizeof(double) * n);
    return LBM_OK;
}

lbm_status lbm_get_history(lbm_ctx* c, double* host_out, int max_entries, int* n_out) {
    CHECK_CTX(c);
    if (!host_out || max_entries < 0) return fail(c, LBM_ERR_INVALID_ARG, "bad output buffer");
    if (!c->started) return fail(c, LBM_ERR_STATE, "no solve state");
    CUDA_TRY(c, cudaSetDevice(c->device));
    lbm_status st = read_ctl(c, c->stream);
    if (st != LBM_OK) return st;
    const long long checks = c->h_ctl->checks;
    const long long kept = checks < kHistCap ? checks : kHistCap;
    const long long n = kept < max_entries ? kept : max_entries;
    std::vector<double> ring(4 * (size_t)kHistCap);
    if (n > 0)
        CUDA_TRY(c, cudaMemcpy(ring.data(), c->d_hist, sizeof(double) * 4 * kHistCap,
                               cudaMemcpyDeviceToHost));
    // the n most recent checks, oldest first
    for (long long i = 0; i < n; ++i) {
        const long long chk = checks - n + i;           // 0-based check index
        std::memcpy(host_out + 4 * i, &ring[4 * (size_t)(chk % kHistCap)], sizeof(double) * 4);
    }
    if (n_out) *n_out = (int)n;
    return LBM_OK;
}

// ---- checkpoint / resume ----
// A snapshot holds everything the iteration carries from one step to the
// next: the current distributions, the reference frames, the temperature
// snapshot of the residual, the control block (iteration count, residual
// bookkeeping), the check history and the last plane fluxes, behind a header
// that names the solve it belongs to.
namespace {

struct StateHeader {
    char magic[8];                         // "MRTLBMS2": four stored fields per node
    int32_t n[3], axis, lateral, fmt, NX, NY, NZ, pitch, check_every, pad;
    double s, t_hot, t_cold;
    int64_t f_bytes, cells;
};

size_t state_bytes(const lbm_ctx* c) {
    const size_t esize = c->fmt == LBM_STORE_F32 ? 4 : 2;
    const size_t cells = (size_t)c->pstride;
    return sizeof(StateHeader) + lbm::kFields * cells * esize + sizeof(float) * 5 * (size_t)c->L.NZ +
           sizeof(float) * cells + sizeof(Ctl) + sizeof(double) * 4 * kHistCap +
           sizeof(double) * (size_t)c->L.NZ;
}

StateHeader state_header(const lbm_ctx* c) {
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "MRTLBMS2", 8);
    for (int i = 0; i < 3; ++i) h.n[i] = c->n[i];
    h.axis = c->axis;
    h.lateral = c->lateral;
    h.fmt = c->fmt;
    h.NX = c->L.NX;
    h.NY = c->L.NY;
    h.NZ = c->L.NZ;
    h.pitch = c->L.pitch;
    h.check_every = c->opts.check_every;
    h.s = c->s;
    h.t_hot = c->opts.t_hot;
    h.t_cold = c->opts.t_cold;
    h.cells = c->pstride;
    h.f_bytes = lbm::kFields * c->pstride * (c->fmt == LBM_STORE_F32 ? 4 : 2);
    return h;
}

}  // namespace

size_t lbm_state_bytes(const lbm_ctx* c) {
    if (!c || c->poisoned || !c->started) return 0;
    return state_bytes(c);
}

lbm_status lbm_get_state(lbm_ctx* c, void* host_out, size_t bytes) {
    CHECK_CTX(c);
    if (!c->started) return fail(c, LBM_ERR_STATE, "no solve state to save");
    if (!host_out || bytes < state_bytes(c))
        return fail(c, LBM_ERR_INVALID_ARG, "host_out must hold lbm_state_bytes() = %zu bytes",
                    state_bytes(c));
    CUDA_TRY(c, cudaSetDevice(c->device));
    const StateHeader h = state_header(c);
    char* p = static_cast<char*>(host_out);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    cudaStream_t st = c->stream;
    const size_t cells = (size_t)c->pstride;
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_f[c->cur], (size_t)h.f_bytes, cudaMemcpyDeviceToHost, st));
    p += h.f_bytes;
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_ref, sizeof(float) * 5 * c->L.NZ, cudaMemcpyDeviceToHost, st));
    p += sizeof(float) * 5 * c->L.NZ;
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_tsnap, sizeof(float) * cells, cudaMemcpyDeviceToHost, st));
    p += sizeof(float) * cells;
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    p += sizeof(Ctl);
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_hist, sizeof(double) * 4 * kHistCap, cudaMemcpyDeviceToHost, st));
    p += sizeof(double) * 4 * kHistCap;
    CUDA_TRY(c, cudaMemcpyAsync(p, c->d_Q, sizeof(double) * c->L.NZ, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(c, cudaStreamSynchronize(st));
    return LBM_OK;
}

lbm_status lbm_set_state(lbm_ctx* c, const void* host_in, size_t bytes) {
    CHECK_CTX(c);
    if (!c->started) return fail(c, LBM_ERR_STATE, "call lbm_start for the same solve first");
    if (!host_in || bytes < sizeof(StateHeader))
        return fail(c, LBM_ERR_INVALID_ARG, "host_in is NULL or too short");
    StateHeader h;
    std::memcpy(&h, host_in, sizeof h);
    const StateHeader want = state_header(c);
    if (std::memcmp(h.magic, want.magic, 8) != 0)
        return fail(c, LBM_ERR_INVALID_ARG, "not a solver state snapshot");
    if (std::memcmp(&h, &want, sizeof h) != 0)
        return fail(c, LBM_ERR_INVALID_ARG, "the snapshot belongs to another solve (cell size, axis, "
                                            "lateral type, storage, check interval, walls or scale differ)");
    if (bytes < state_bytes(c)) return fail(c, LBM_ERR_INVALID_ARG, "the snapshot is truncated");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const char* p = static_cast<const char*>(host_in) + sizeof h;
    cudaStream_t st = c->stream;
    const size_t cells = (size_t)c->pstride;
    c->cur = 0;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_f[0], p, (size_t)h.f_bytes, cudaMemcpyHostToDevice, st));
    p += h.f_bytes;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ref, p, sizeof(float) * 5 * c->L.NZ, cudaMemcpyHostToDevice, st));
    p += sizeof(float) * 5 * c->L.NZ;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_tsnap, p, sizeof(float) * cells, cudaMemcpyHostToDevice, st));
    p += sizeof(float) * cells;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_ctl, p, sizeof(Ctl), cudaMemcpyHostToDevice, st));
    p += sizeof(Ctl);
    CUDA_TRY(c, cudaMemcpyAsync(c->d_hist, p, sizeof(double) * 4 * kHistCap, cudaMemcpyHostToDevice, st));
    p += sizeof(double) * 4 * kHistCap;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_Q, p, sizeof(double) * c->L.NZ, cudaMemcpyHostToDevice, st));
    CUDA_TRY(c, cudaMemsetAsync(c->d_plane_cnt, 0, sizeof(int) * c->L.NZ, st));
    lbm_status s2 = read_ctl(c, st);
    if (s2 != LBM_OK) return s2;
    return LBM_OK;
}

int lbm_debug_build(void) {
#ifdef LBM_DEBUG
    return 1;
#else
    return 0;
#endif
}

lbm_status lbm_debug_error(unsigned* out, int clear) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = 0;
#ifdef LBM_DEBUG
    if (cudaMemcpyFromSymbol(out, lbm::g_lbm_debug, sizeof *out) != cudaSuccess) return LBM_ERR_CUDA;
    if (clear) {
        const unsigned z = 0;
        if (cudaMemcpyToSymbol(lbm::g_lbm_debug, &z, sizeof z) != cudaSuccess) return LBM_ERR_CUDA;
    }
#else
    (void)clear;
#endif
    return LBM_OK;
}

lbm_status lbm_get_launch_plan(const lbm_ctx* c, lbm_launch_plan* out) {
    if (!c || !out) return LBM_ERR_INVALID_ARG;
    if (!c->started) return LBM_ERR_STATE;
    std::memset(out, 0, sizeof *out);
    out->nx = c->L.NX;
    out->ny = c->L.NY;
    out->nz = c->L.NZ;
    out->pitch = c->L.pitch;
    out->steps_per_launch = fusable(c) ? 2 : 1;
    if (fusable(c)) {
        out->tile_rows = c->f2.fy;
        out->zchunk = c->f2.zchunk;
        out->block_threads = c->f2.threads;
    }
    return LBM_OK;
}

lbm_status lbm_get_geometry(lbm_ctx* c, uint8_t* host_out) {
    CHECK_CTX(c);
    if (!host_out) return fail(c, LBM_ERR_INVALID_ARG, "host_out is NULL");
    if (!c->have_geometry) return fail(c, LBM_ERR_STATE, "no geometry set");
    CUDA_TRY(c, cudaSetDevice(c->device));
    const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    CUDA_TRY(c, cudaMemcpy(host_out, c->d_phase, N, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

lbm_status lbm_yarn_conductivity(double lam_fL, double lam_fT, double lam_m, double phi_fy,
                                 double* lam_L, double* lam_T) {
    if (!(lam_fL > 0.0) || !(lam_fT > 0.0) || !(lam_m > 0.0) || !(phi_fy > 0.0) ||
        !(phi_fy < 1.0) || lam_fT == lam_m)
        return LBM_ERR_INVALID_ARG;
    if (lam_L) *lam_L = lam_fL * phi_fy + lam_m * (1.0 - phi_fy);
    if (lam_T) *lam_T = lam_m + phi_fy / (1.0 / (lam_fT - lam_m) + (1.0 - phi_fy) / (2.0 * lam_m));
    return LBM_OK;
}

lbm_status lbm_braid_unit_cell(double phi_f, int n_f, double d_f, double gamma_rad, double* a,
                               double* h, double* c, double* d, double* phi_fy) {
    const double pi = 3.14159265358979323846;
    const double phi_y = pi * std::sqrt(3.0) / 8.0;
    if (!(phi_f > 0.0) || !(phi_f < phi_y) || n_f < 1 || !(d_f > 0.0) || !(gamma_rad > 0.0) ||
        !(gamma_rad < pi / 2))
        return LBM_ERR_INVALID_ARG;
    const double pfy = phi_f / phi_y;
    const double area = (double)n_f * pi * d_f * d_f / 4.0 / pfy;
    const double cg = std::cos(gamma_rad);
    const double dd = std::sqrt(area / (pi * std::sqrt(3.0) * cg));
    const double cc = dd * std::sqrt(3.0) * cg;
    const double aa = 8.0 * dd;
    if (a) *a = aa;
    if (h) *h = aa / std::tan(gamma_rad);
    if (c) *c = cc;
    if (d) *d = dd;
    if (phi_fy) *phi_fy = pfy;
    return LBM_OK;
}

const char* lbm_last_error(const lbm_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_graphs(c);
    if (!c->ws) {                           // a workspace stays the caller's
        cudaFree(c->d_f[0]);
        cudaFree(c->d_f[1]);
        cudaFree(c->d_phase_c);
        cudaFree(c->d_tsnap);
        cudaFree(c->d_ref);
        cudaFree(c->d_sb);
        cudaFree(c->d_part);
        cudaFree(c->d_Q);
        cudaFree(c->d_plane_cnt);
        cudaFree(c->d_T);
        cudaFree(c->d_phase);
        cudaFree(c->d_ctl);
        cudaFree(c->d_hist);
    }
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    cudaGetLastError();
    delete c;
}

// Internal hooks for the voxeliser translation unit (hidden, not part of the ABI).
#define LBM_HIDDEN __attribute__((visibility("hidden")))
LBM_HIDDEN uint8_t* lbm__device_phase(lbm_ctx* c) { return c ? c->d_phase : nullptr; }
LBM_HIDDEN int lbm__dims(const lbm_ctx* c, int* n) {
    if (!c) return -1;
    n[0] = c->n[0]; n[1] = c->n[1]; n[2] = c->n[2];
    return c->device;
}
LBM_HIDDEN void lbm__set_phase_count(lbm_ctx* c, int n_phases) {
    if (c->have_tensors && (int)c->lambda.size() != 6 * n_phases) c->have_tensors = false;
    c->n_phases = n_phases;
    c->have_geometry = true;
    c->started = false;
}
LBM_HIDDEN void lbm__set_error(lbm_ctx* c, const char* msg) { if (c) c->err = msg; }
LBM_HIDDEN int lbm__poisoned(const lbm_ctx* c) { return c ? (c->poisoned ? 1 : 0) : 1; }
LBM_HIDDEN void lbm__poison(lbm_ctx* c) { if (c) c->poisoned = true; }
// Voxeliser scratch inside a workspace (returns 0 for a context without one).
LBM_HIDDEN int lbm__voxel_scratch(lbm_ctx* c, int n_max, double2** anchors, unsigned long long** hist) {
    if (!c || !c->ws || n_max > kWsYarns) return 0;
    *anchors = c->d_vox_anchor;
    *hist = c->d_vox_hist;
    return 1;
}

}  // extern "C"
