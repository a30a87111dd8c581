// Batched solver: many independent cells (different sizes, materials and
// directions) advanced together by one CUDA graph launch.
//
// The paper's application is a sweep over fibre fraction, braiding angle and
// direction (Section 5, Fig. 9); each point is an independent steady solve.
// All solves of a batch are resident in HBM at once.  One batched step launch
// covers every active solve: block b finds its solve by a binary search in a
// per-solve prefix of block counts, loads that solve's descriptor into shared
// memory and runs the same fused step as the single-solve kernel.  Check
// steps close per solve (plane and solve tickets, as in the single-solve
// path); a one-block control kernel then drops converged solves from the
// prefix (so their blocks are no longer launched work) and sets the graph's
// while condition.  The block size is chosen by timing the candidates on the
// batch itself before the solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "lbm.h"
#include "lbm_kernels.cuh"

namespace {

using lbm::Ctl;
using lbm::Layout;
using lbm::StepArgs;

struct BatchDesc {
    StepArgs a;          // src/dst/rsrc/rdst are filled in per launch
    void* f[2];          // distribution buffers
    float* ref;          // frames R_a, R_b, R_c, init tables [5][NZ]
    int blocks;          // blocks of one single step = blocks_per_plane * NZ
    int blocks2;         // blocks of one two-step launch (tiles x z chunks), 0 without
};

// argument variants per solve: buffer parity (2) x reference frame (AA, AB, BB)
constexpr int kVariants = 6;

struct BatchCtl {
    int n_active;        // solves still iterating
    int total_blocks;    // blocks of the active solves
    unsigned long long t0;   // device time (ns) when the solve's graph launch began
};

constexpr int kBatchHistCap = 4096;   // checks kept per solve

// Records the device time at which the batch's iteration starts.
__global__ void batch_stamp_kernel(BatchCtl* bctl) { bctl->t0 = lbm::globaltimer_ns(); }

// Block -> solve: prefix[s] = first block of the s-th active solve, order[s]
// its solve index; prefix[n_active] = total.  Each solve has one ready-made
// argument block per (buffer parity, reference frame), so a block only
// searches the prefix and then reads its arguments through the cache.
template <int FMT, bool PERIODIC, bool CHECK, int THREADS>
__global__ void __launch_bounds__(THREADS, (CHECK && FMT != 0) ? 512 / THREADS : 1024 / THREADS)
batch_step_kernel(const StepArgs* __restrict__ args, const int* __restrict__ prefix,
                  const int* __restrict__ order, const BatchCtl* __restrict__ bctl, int variant,
                  unsigned rseed) {
    const int n_active = bctl->n_active;
    const int total = prefix[n_active];
    if ((int)blockIdx.x >= total) return;     // block of a solve that has converged
    // odd steps walk the blocks backwards, so that a step starts on the state
    // the previous one wrote last (still in L2)
    const int b = (rseed & 1u) ? total - 1 - (int)blockIdx.x : (int)blockIdx.x;
    int lo = 0, hi = n_active - 1;            // last s with prefix[s] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const StepArgs& a = args[order[lo] * kVariants + variant];
    const int local = b - prefix[lo];
    const int z = local / a.blocks_per_plane;
    // rows without padding skip the ragged-row handling (block-uniform branch)
    if (a.nx == a.pitch)
        lbm::step_body<FMT, PERIODIC, CHECK, false, THREADS>(a, local - z * a.blocks_per_plane, z, rseed);
    else
        lbm::step_body<FMT, PERIODIC, CHECK, true, THREADS>(a, local - z * a.blocks_per_plane, z, rseed);
}

// Two fused FP32 steps per launch over every active solve: block b finds its
// solve in the prefix of two-step block counts and runs one tile (f2_fy rows,
// f2_zchunk planes) of the single-solve two-step kernel's body.  Every block
// of the launch has the same size; a solve whose rows hold fewer threads
// leaves the rest idle.  flip reverses the block order and the chunks'
// marching direction on alternate launches (a launch starts on what the
// previous one wrote last).
template <bool PERIODIC>
__global__ void __launch_bounds__(lbm::F2_MAX_THREADS, 1)
batch_fused2_kernel(const StepArgs* __restrict__ args, const int* __restrict__ prefix2,
                    const int* __restrict__ order, const BatchCtl* __restrict__ bctl, int variant, int flip) {
    const int n_active = bctl->n_active;
    const int total = prefix2[n_active];
    if ((int)blockIdx.x >= total) return;     // block of a solve that has converged
    const int b = flip ? total - 1 - (int)blockIdx.x : (int)blockIdx.x;
    int lo = 0, hi = n_active - 1;            // last s with prefix2[s] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix2[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    const StepArgs& a = args[order[lo] * kVariants + variant];
    const int local = b - prefix2[lo];
    const int bz = local / a.f2_bxy;
    const int by = local - bz * a.f2_bxy;
    float4* s_sa;
    float2* s_sc;
    float* fn = lbm::fused2_tables(a, 3 * lbm::f2_slot_rows(a.f2_fy) * a.pitch, &s_sa, &s_sc);
    lbm::fused2_body<PERIODIC, 0>(a, fn, s_sa, s_sc, a.f2_fy, by, bz, a.f2_zchunk, flip);
}

// After a check: keep the solves that are not done, rebuild the prefixes and
// set the while condition (any solve still active).
__global__ void batch_control_kernel(const BatchDesc* __restrict__ descs, int n_solves,
                                     int* __restrict__ prefix, int* __restrict__ prefix2,
                                     int* __restrict__ order, BatchCtl* __restrict__ bctl,
                                     cudaGraphConditionalHandle handle, int use_handle) {
    if (threadIdx.x != 0) return;
    int n = 0, total = 0, total2 = 0;
    for (int s = 0; s < n_solves; ++s) {
        const Ctl* c = descs[s].a.ck.ctl;
        if (c->done) continue;
        order[n] = s;
        prefix[n] = total;
        prefix2[n] = total2;
        total += descs[s].blocks;
        total2 += descs[s].blocks2;
        ++n;
    }
    prefix[n] = total;
    prefix2[n] = total2;
    bctl->n_active = n;
    bctl->total_blocks = total;
    if (use_handle) cudaGraphSetConditional(handle, n > 0 ? 1u : 0u);
}

struct Cell {
    int n[3];
    int axis;
    int n_phases;
    std::vector<uint8_t> phase;
    std::vector<double> lambda;
    std::vector<float> t_init;     // initial temperature (original order) or empty
};

}  // namespace

struct lbm_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::string err;
    bool poisoned = false;
    std::vector<Cell> cells;
    // device state of the last solve
    char* arena = nullptr;
    size_t arena_bytes = 0;
    BatchDesc* d_descs = nullptr;          // per solve: blocks and the control block
    StepArgs* d_args = nullptr;            // per solve: kVariants argument blocks
    std::vector<BatchDesc> descs;
    std::vector<Layout> layouts;
    std::vector<double> scale;             // lattice scale s per solve
    int* d_prefix = nullptr;
    int* d_prefix2 = nullptr;              // prefix of two-step block counts
    int* d_order = nullptr;
    BatchCtl* d_bctl = nullptr;
    Ctl* h_ctl = nullptr;                  // pinned, one per solve
    int fmt = 0, lateral = 0, threads = 256, K = 100;
    int max_blocks = 0, max_phases = 1;
    bool fused = false;                    // plain steps as two-step launches
    int f2_threads = 0, max_blocks2 = 0;
    size_t f2_smem = 0;
    int cur = 0;
    bool solved = false;
    lbm_solve_opts opts{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    return st;
}

#define BCUDA(b, call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            (b)->poisoned = true;                                                           \
            return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OUT_OF_MEMORY      \
                                                              : LBM_ERR_CUDA,               \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                   \
        }                                                                                   \
    } while (0)

void free_device(lbm_batch* b) {
    cudaFree(b->arena);
    cudaFree(b->d_descs);
    cudaFree(b->d_args);
    cudaFree(b->d_prefix);
    cudaFree(b->d_prefix2);
    cudaFree(b->d_order);
    cudaFree(b->d_bctl);
    if (b->h_ctl) cudaFreeHost(b->h_ctl);
    b->arena = nullptr;
    b->d_descs = nullptr;
    b->d_args = nullptr;
    b->d_prefix = b->d_prefix2 = b->d_order = nullptr;
    b->d_bctl = nullptr;
    b->h_ctl = nullptr;
    b->arena_bytes = 0;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Launch {
    bool check;
    int parity, frame;
    unsigned rseed;
};

template <int FMT, bool PERIODIC, int THREADS>
void launch_batch(const lbm_batch* b, const Launch& l, cudaStream_t st) {
    const size_t smem = sizeof(float4) * 2 * b->max_phases;
    const int variant = l.parity * 3 + l.frame;
    if (l.check)
        batch_step_kernel<FMT, PERIODIC, true, THREADS><<<b->max_blocks, THREADS, smem, st>>>(
            b->d_args, b->d_prefix, b->d_order, b->d_bctl, variant, l.rseed);
    else
        batch_step_kernel<FMT, PERIODIC, false, THREADS><<<b->max_blocks, THREADS, smem, st>>>(
            b->d_args, b->d_prefix, b->d_order, b->d_bctl, variant, l.rseed);
}

template <int FMT>
void launch_fmt(const lbm_batch* b, const Launch& l, cudaStream_t st) {
    const bool per = b->lateral == LBM_LATERAL_PERIODIC;
    switch (b->threads) {
        case 128:
            per ? launch_batch<FMT, true, 128>(b, l, st) : launch_batch<FMT, false, 128>(b, l, st);
            break;
        case 512:
            per ? launch_batch<FMT, true, 512>(b, l, st) : launch_batch<FMT, false, 512>(b, l, st);
            break;
        default:
            per ? launch_batch<FMT, true, 256>(b, l, st) : launch_batch<FMT, false, 256>(b, l, st);
    }
}

cudaError_t launch_step(const lbm_batch* b, bool check, int parity, int frame, unsigned rseed,
                        cudaStream_t st) {
    const Launch l{check, parity, frame, rseed};
    if (b->fmt == LBM_STORE_BF16) launch_fmt<1>(b, l, st);
    else if (b->fmt == LBM_STORE_F16) launch_fmt<2>(b, l, st);
    else launch_fmt<0>(b, l, st);
    return cudaGetLastError();
}

// Two FP32 steps of every active solve (state in buffer `parity`, frame BB).
cudaError_t launch_pair(const lbm_batch* b, int parity, int flip, cudaStream_t st) {
    const int variant = parity * 3 + 2;
    if (b->lateral == LBM_LATERAL_PERIODIC)
        batch_fused2_kernel<true><<<b->max_blocks2, b->f2_threads, b->f2_smem, st>>>(
            b->d_args, b->d_prefix2, b->d_order, b->d_bctl, variant, flip);
    else
        batch_fused2_kernel<false><<<b->max_blocks2, b->f2_threads, b->f2_smem, st>>>(
            b->d_args, b->d_prefix2, b->d_order, b->d_bctl, variant, flip);
    return cudaGetLastError();
}

// Tile of a solve's two-step launch with blocks of `threads` threads: the
// tallest tile whose rows fit the block.  False if the rows are not a
// multiple of 4 nodes or a row needs more than a third of the block.
bool f2_tile(int nx, int ny, int threads, int* fy, int* bxy) {
    if (nx % 4) return false;
    const int rows = threads / (nx / 4);
    if (rows < 3) return false;
    *fy = rows - 2;
    *bxy = (ny + *fy - 1) / *fy;
    return true;
}

// Lays out one solve inside the arena and writes its descriptor.
struct Plan {
    size_t off_f[2], off_phase, off_tsnap, off_ref, off_part, off_Q, off_cnt, off_ctl, off_sb;
    size_t off_hist, off_hist_t;
    size_t bytes;
};

Plan plan_solve(const Layout& L, int n_phases, size_t esize, int bpp, size_t base) {
    Plan p;
    const size_t cells = (size_t)L.pitch * L.NY * L.NZ;
    size_t o = base;
    p.off_f[0] = o; o = align256(o + lbm::kFields * cells * esize);
    p.off_f[1] = o; o = align256(o + lbm::kFields * cells * esize);
    p.off_phase = o; o = align256(o + cells);
    p.off_tsnap = o; o = align256(o + cells * sizeof(float));
    p.off_ref = o; o = align256(o + 5 * (size_t)L.NZ * sizeof(float));
    p.off_part = o; o = align256(o + 4 * (size_t)L.NZ * bpp * sizeof(double));
    p.off_Q = o; o = align256(o + 3 * (size_t)L.NZ * sizeof(double));
    p.off_cnt = o; o = align256(o + (size_t)L.NZ * sizeof(int));
    p.off_ctl = o; o = align256(o + sizeof(Ctl));
    p.off_sb = o; o = align256(o + 2 * (size_t)n_phases * sizeof(float4));
    p.off_hist = o; o = align256(o + 4 * (size_t)kBatchHistCap * sizeof(double));
    p.off_hist_t = o; o = align256(o + (size_t)kBatchHistCap * sizeof(unsigned long long));
    p.bytes = o - base;
    return p;
}

int grid_1d(long long total) {
    long long g = (total + 255) / 256;
    if (g > 152LL * 32) g = 152LL * 32;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(int cuda_device, lbm_batch** out) {
    if (!out) return LBM_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cuda_device < 0 || cuda_device >= ndev) {
        cudaGetLastError();
        return LBM_ERR_INVALID_ARG;
    }
    lbm_batch* b = new (std::nothrow) lbm_batch();
    if (!b) return LBM_ERR_OUT_OF_MEMORY;
    b->device = cuda_device;
    lbm_default_opts(&b->opts);
    if (cudaSetDevice(cuda_device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&b->ev0) != cudaSuccess || cudaEventCreate(&b->ev1) != cudaSuccess) {
        cudaGetLastError();
        lbm_batch_destroy(b);
        return LBM_ERR_CUDA;
    }
    *out = b;
    return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch* b, int nx, int ny, int nz, const uint8_t* phase, int n_phases,
                         const double* lambda, lbm_axis axis, int* id) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (b->poisoned) return bfail(b, LBM_ERR_CUDA, "batch poisoned by an earlier CUDA error");
    if (nx < 2 || ny < 2 || nz < 2 || (long long)nx * ny * nz >= (1LL << 31))
        return bfail(b, LBM_ERR_INVALID_ARG, "sizes must be >= 2 with nx*ny*nz < 2^31");
    if (!phase || !lambda || n_phases < 1 || n_phases > 255)
        return bfail(b, LBM_ERR_INVALID_ARG, "need a phase map, tensors and 1 <= n_phases <= 255");
    if (axis < LBM_AXIS_X || axis > LBM_AXIS_Z) return bfail(b, LBM_ERR_INVALID_ARG, "bad axis");
    const size_t N = (size_t)nx * ny * nz;
    for (size_t i = 0; i < N; ++i)
        if (phase[i] >= n_phases)
            return bfail(b, LBM_ERR_INVALID_ARG, "phase id %d at voxel %zu >= n_phases", (int)phase[i], i);
    for (int p = 0; p < n_phases; ++p) {
        const double* t = lambda + 6 * p;
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(t[k])) return bfail(b, LBM_ERR_INVALID_ARG, "tensor %d not finite", p);
        // Cholesky test (symmetric positive definite)
        const double l00 = t[0] > 0 ? std::sqrt(t[0]) : -1;
        if (!(l00 > 0)) return bfail(b, LBM_ERR_INVALID_ARG, "tensor %d not positive definite", p);
        const double l10 = t[5] / l00, l20 = t[4] / l00;
        const double d1 = t[1] - l10 * l10;
        if (!(d1 > 0)) return bfail(b, LBM_ERR_INVALID_ARG, "tensor %d not positive definite", p);
        const double l21 = (t[3] - l20 * l10) / std::sqrt(d1);
        if (!(t[2] - l20 * l20 - l21 * l21 > 0))
            return bfail(b, LBM_ERR_INVALID_ARG, "tensor %d not positive definite", p);
    }
    Cell c;
    c.n[0] = nx;
    c.n[1] = ny;
    c.n[2] = nz;
    c.axis = axis;
    c.n_phases = n_phases;
    c.phase.assign(phase, phase + N);
    c.lambda.assign(lambda, lambda + 6 * n_phases);
    b->cells.push_back(std::move(c));
    b->solved = false;
    if (id) *id = (int)b->cells.size() - 1;
    return LBM_OK;
}

lbm_status lbm_batch_solve(lbm_batch* b, lbm_lateral lateral, const lbm_solve_opts* o,
                           lbm_batch_info* info) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (b->poisoned) return bfail(b, LBM_ERR_CUDA, "batch poisoned by an earlier CUDA error");
    if (b->cells.empty()) return bfail(b, LBM_ERR_STATE, "no solves added");
    if (lateral != LBM_LATERAL_PERIODIC && lateral != LBM_LATERAL_ADIABATIC)
        return bfail(b, LBM_ERR_INVALID_ARG, "bad lateral type");
    lbm_solve_opts op;
    if (o) op = *o;
    else lbm_default_opts(&op);
    if (!(op.t_hot != op.t_cold) || op.check_every < 2 || (op.check_every & 1) ||
        op.check_every > 4096 || op.max_iters < 0 || op.t_init ||
        (op.storage != LBM_STORE_F32 && op.storage != LBM_STORE_BF16 && op.storage != LBM_STORE_F16) ||
        (!(op.lattice_scale > 0.0) && !(op.tau_max > 0.5)))
        return bfail(b, LBM_ERR_INVALID_ARG,
                     "invalid options (walls, even check_every <= 4096, storage, tau_max; no t_init)");
    BCUDA(b, cudaSetDevice(b->device));
    nvtxRangePushA("lbm_batch_solve");
    struct PopOnExit {
        ~PopOnExit() { nvtxRangePop(); }
    } pop_on_exit;
    free_device(b);
    b->opts = op;
    b->fmt = op.storage;
    b->lateral = lateral;
    b->K = op.check_every;
    const int V = op.storage == LBM_STORE_F32 ? 4 : 8;
    const size_t esize = op.storage == LBM_STORE_F32 ? 4 : 2;
    const int n_solves = (int)b->cells.size();
    const double eps = 0.25;
    const double t_ref = 0.5 * (op.t_hot + op.t_cold);
    int e2 = 0;
    std::frexp(std::fmax(std::fmax(std::fabs(op.t_hot), std::fabs(op.t_cold)), 1.0), &e2);
    const double quantum = std::ldexp(1.0, e2 - 20);
    static const int perms[3][3] = {{1, 2, 0}, {2, 0, 1}, {0, 1, 2}};

    // the scratch of the check partials grows with the number of blocks per
    // plane: plan for the smallest candidate block size (128 threads)
    std::vector<Plan> plans(n_solves);
    b->layouts.assign(n_solves, Layout{});
    size_t total = 0;
    b->max_phases = 1;
    for (int s = 0; s < n_solves; ++s) {
        const Cell& c = b->cells[s];
        Layout& L = b->layouts[s];
        for (int i = 0; i < 3; ++i) {
            L.n[i] = c.n[i];
            L.perm[i] = perms[c.axis][i];
        }
        // FP32 storage: order the lateral axes so that rows are a multiple
        // of 4 nodes (two-step launches need it) and as short as possible
        // (taller tiles per block); the relabelling is exact
        if (op.storage == LBM_STORE_F32) {
            const int a0 = c.n[L.perm[0]], a1 = c.n[L.perm[1]];
            const bool ok0 = a0 % 4 == 0, ok1 = a1 % 4 == 0;
            if ((ok1 && !ok0) || (ok0 && ok1 && a1 < a0)) std::swap(L.perm[0], L.perm[1]);
        }
        L.NX = c.n[L.perm[0]];
        L.NY = c.n[L.perm[1]];
        L.NZ = c.n[L.perm[2]];
        L.pitch = (L.NX + V - 1) / V * V;
        if (L.NZ > 65535) return bfail(b, LBM_ERR_INVALID_ARG, "axis longer than 65535 nodes");
        const int quads = (L.pitch / V) * L.NY;
        const int bpp_max = (quads + 127) / 128;   // smallest candidate block size
        plans[s] = plan_solve(L, c.n_phases, esize, bpp_max, total);
        total += plans[s].bytes;
        b->max_phases = std::max(b->max_phases, c.n_phases);
    }
    BCUDA(b, cudaMalloc((void**)&b->arena, total));
    b->arena_bytes = total;
    BCUDA(b, cudaMalloc((void**)&b->d_descs, sizeof(BatchDesc) * n_solves));
    BCUDA(b, cudaMalloc((void**)&b->d_args, sizeof(StepArgs) * kVariants * n_solves));
    BCUDA(b, cudaMalloc((void**)&b->d_prefix, sizeof(int) * (n_solves + 1)));
    BCUDA(b, cudaMalloc((void**)&b->d_prefix2, sizeof(int) * (n_solves + 1)));
    BCUDA(b, cudaMalloc((void**)&b->d_order, sizeof(int) * n_solves));
    BCUDA(b, cudaMalloc((void**)&b->d_bctl, sizeof(BatchCtl)));
    BCUDA(b, cudaMallocHost((void**)&b->h_ctl, sizeof(Ctl) * n_solves));

    // per solve: geometry (permuted on the device), S_b = tau^-1, frames, init
    uint8_t* d_stage = nullptr;
    float* d_tstage = nullptr;
    size_t max_cells = 0, max_init = 0;
    for (auto& c : b->cells) {
        max_cells = std::max(max_cells, c.phase.size());
        max_init = std::max(max_init, c.t_init.size());
    }
    BCUDA(b, cudaMalloc((void**)&d_stage, max_cells));
    if (max_init) BCUDA(b, cudaMalloc((void**)&d_tstage, sizeof(float) * max_init));
    b->descs.assign(n_solves, BatchDesc{});
    b->scale.assign(n_solves, 0.0);
    cudaStream_t st = b->stream;
    for (int s = 0; s < n_solves; ++s) {
        const Cell& c = b->cells[s];
        const Layout& L = b->layouts[s];
        const Plan& p = plans[s];
        char* base = b->arena;
        double smax = op.lattice_scale;
        if (!(smax > 0.0)) {
            double m = 0.0;
            for (int q = 0; q < c.n_phases; ++q)
                for (int k = 0; k < 3; ++k) m = std::fmax(m, c.lambda[6 * q + k]);
            smax = eps * (op.tau_max - 0.5) / m;
        }
        const double sc = smax;
        b->scale[s] = sc;
        std::vector<float4> sb(2 * (size_t)c.n_phases);
        for (int q = 0; q < c.n_phases; ++q) {
            const double* t = &c.lambda[6 * q];
            const double full[9] = {t[0], t[5], t[4], t[5], t[1], t[3], t[4], t[3], t[2]};
            double tau[9], S[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    tau[3 * i + j] = sc * full[3 * L.perm[i] + L.perm[j]] / eps + (i == j ? 0.5 : 0.0);
            const double c00 = tau[4] * tau[8] - tau[5] * tau[7];
            const double c01 = tau[5] * tau[6] - tau[3] * tau[8];
            const double c02 = tau[3] * tau[7] - tau[4] * tau[6];
            const double det = tau[0] * c00 + tau[1] * c01 + tau[2] * c02;
            S[0] = c00 / det;
            S[1] = (tau[2] * tau[7] - tau[1] * tau[8]) / det;
            S[2] = (tau[1] * tau[5] - tau[2] * tau[4]) / det;
            S[4] = (tau[0] * tau[8] - tau[2] * tau[6]) / det;
            S[5] = (tau[2] * tau[3] - tau[0] * tau[5]) / det;
            S[8] = (tau[0] * tau[4] - tau[1] * tau[3]) / det;
            // the device's per-phase table: B = (I - S_b) / 2 for FP32, S_b for 16 bits
            lbm::phase_entry(S, &sb[2 * (size_t)q]);
        }
        BCUDA(b, cudaMemcpyAsync(base + p.off_sb, sb.data(), sizeof(float4) * sb.size(),
                                 cudaMemcpyHostToDevice, st));
        // initial frame: the plane means of the initial field on the
        // quantum grid (the linear profile, or the solve's own start field)
        std::vector<double> mean(L.NZ, 0.0);
        if (!c.t_init.empty()) {
            const size_t N = c.t_init.size();
            for (size_t i = 0; i < N; ++i) {
                const int cc[3] = {(int)(i % c.n[0]), (int)((i / c.n[0]) % c.n[1]),
                                   (int)(i / ((size_t)c.n[0] * c.n[1]))};
                mean[cc[L.perm[2]]] += c.t_init[i];
            }
            for (auto& m : mean) m /= (double)L.NX * (double)L.NY;
        } else {
            for (int z = 0; z < L.NZ; ++z)
                mean[z] = op.t_hot + (op.t_cold - op.t_hot) * ((double)z + 0.5) / (double)L.NZ;
        }
        std::vector<float> ref(5 * (size_t)L.NZ);
        for (int z = 0; z < L.NZ; ++z) {
            const double T0 = op.t_hot + (op.t_cold - op.t_hot) * ((double)z + 0.5) / (double)L.NZ;
            const double r = std::nearbyint(mean[z] / quantum) * quantum;
            ref[z] = ref[L.NZ + z] = ref[2 * L.NZ + z] = (float)r;
            ref[3 * L.NZ + z] = (float)(T0 - r);
            ref[4 * L.NZ + z] = (float)(T0 - t_ref);
        }
        const float* tinit = nullptr;
        if (!c.t_init.empty()) {
            BCUDA(b, cudaMemcpyAsync(d_tstage, c.t_init.data(), sizeof(float) * c.t_init.size(),
                                     cudaMemcpyHostToDevice, st));
            tinit = d_tstage;
        }
        float* d_ref = reinterpret_cast<float*>(base + p.off_ref);
        BCUDA(b, cudaMemcpyAsync(d_ref, ref.data(), sizeof(float) * ref.size(), cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(d_stage, c.phase.data(), c.phase.size(), cudaMemcpyHostToDevice, st));
        const long long cells = (long long)L.pitch * L.NY * L.NZ;
        lbm::permute_phase_kernel<<<grid_1d(cells), 256, 0, st>>>(
            d_stage, reinterpret_cast<uint8_t*>(base + p.off_phase), L);
        const float* th = d_ref + 3 * L.NZ;
        const float* ts = d_ref + 4 * L.NZ;
        float* tsnap = reinterpret_cast<float*>(base + p.off_tsnap);
        if (op.storage == LBM_STORE_BF16)
            lbm::init_kernel<1><<<grid_1d(cells), 256, 0, st>>>(base + p.off_f[0], tsnap, cells, L, d_ref,
                                                               th, ts, (float)t_ref, tinit);
        else if (op.storage == LBM_STORE_F16)
            lbm::init_kernel<2><<<grid_1d(cells), 256, 0, st>>>(base + p.off_f[0], tsnap, cells, L, d_ref,
                                                               th, ts, (float)t_ref, tinit);
        else
            lbm::init_kernel<0><<<grid_1d(cells), 256, 0, st>>>(base + p.off_f[0], tsnap, cells, L, d_ref,
                                                               th, ts, (float)t_ref, tinit);
        BCUDA(b, cudaGetLastError());
        BCUDA(b, cudaMemsetAsync(base + p.off_cnt, 0, sizeof(int) * L.NZ, st));
        Ctl h{};
        h.best_rt = INFINITY;
        h.k_eff = h.r_t = h.r_q = NAN;
        h.status = LBM_ERR_NOT_CONVERGED;
        b->h_ctl[s] = h;
        BCUDA(b, cudaMemcpyAsync(base + p.off_ctl, &b->h_ctl[s], sizeof(Ctl), cudaMemcpyHostToDevice, st));
        // the copy must finish before the staging buffer is reused
        BCUDA(b, cudaStreamSynchronize(st));

        BatchDesc& d = b->descs[s];
        std::memset(&d, 0, sizeof d);
        d.f[0] = base + p.off_f[0];
        d.f[1] = base + p.off_f[1];
        d.ref = d_ref;
        StepArgs& a = d.a;
        a.phase = reinterpret_cast<uint8_t*>(base + p.off_phase);
        a.sb = reinterpret_cast<const float4*>(base + p.off_sb);
        a.tsnap = tsnap;
        a.pstride = cells;
        a.nx = L.NX;
        a.ny = L.NY;
        a.nz = L.NZ;
        a.pitch = L.pitch;
        a.n_phases = c.n_phases;
        a.quads_per_plane = (L.pitch / V) * L.NY;
        a.eps_hot = (float)(eps * op.t_hot);
        a.eps_cold = (float)(eps * op.t_cold);
        a.t_ref = t_ref;
        lbm::CheckArgs& k = a.ck;
        k.part = reinterpret_cast<double*>(base + p.off_part);
        k.Q = reinterpret_cast<double*>(base + p.off_Q);
        k.plane = k.Q + L.NZ;
        k.plane_cnt = reinterpret_cast<int*>(base + p.off_cnt);
        k.ctl = reinterpret_cast<Ctl*>(base + p.off_ctl);
        k.ra = d_ref;
        k.rb = d_ref + L.NZ;
        k.rc = d_ref + 2 * L.NZ;
        k.stall_checks = op.stall_checks;
        k.interval = op.check_every;
        k.max_iters = op.max_iters;
        k.tol = op.tol;
        k.keff_scale = (double)L.NZ / (sc * (op.t_hot - op.t_cold) * (double)L.NX * (double)L.NY);
        k.inv_area = 1.0 / ((double)L.NX * (double)L.NY);
        k.quantum = quantum;
        k.inv_quantum = 1.0 / quantum;
        k.hist = reinterpret_cast<double*>(base + p.off_hist);
        k.hist_t = reinterpret_cast<unsigned long long*>(base + p.off_hist_t);
        k.hist_cap = kBatchHistCap;
    }
    cudaFree(d_stage);
    cudaFree(d_tstage);
    b->cur = 0;

    // A launch configuration: single steps with blocks of `threads` threads,
    // and (f2_threads > 0) plain steps as two-step launches with blocks of
    // f2_threads threads and z chunks of about `zc` planes.
    struct Cfg {
        int threads, f2_threads, zc;
    };
    int optin = 0;
    BCUDA(b, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    int n_sm = 152;
    BCUDA(b, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, b->device));
    // per solve two-step tiles for a block size; false if some solve cannot
    auto f2_ok = [&](int t, size_t* smem) {
        *smem = 0;
        for (int s = 0; s < n_solves; ++s) {
            int fy, bxy;
            const Layout& L = b->layouts[s];
            if (L.pitch != L.NX || !f2_tile(L.NX, L.NY, t, &fy, &bxy)) return false;
            *smem = std::max(*smem, lbm::fused2_smem_bytes(L.NX, fy, b->max_phases));
        }
        return *smem + 64 <= (size_t)optin;
    };

    auto upload = [&](const Cfg& cf) -> lbm_status {
        b->threads = cf.threads;
        b->fused = cf.f2_threads > 0;
        b->f2_threads = cf.f2_threads;
        std::vector<int> prefix(n_solves + 1), prefix2(n_solves + 1), order(n_solves);
        int tot = 0, tot2 = 0;
        size_t smem2 = 0;
        for (int s = 0; s < n_solves; ++s) {
            StepArgs& a = b->descs[s].a;
            a.blocks_per_plane = (a.quads_per_plane + cf.threads - 1) / cf.threads;
            b->descs[s].blocks = a.blocks_per_plane * a.nz;
            b->descs[s].blocks2 = 0;
            a.f2_fy = a.f2_bxy = a.f2_zchunk = 0;
            if (b->fused) {
                int fy = 0, bxy = 0;
                f2_tile(a.nx, a.ny, cf.f2_threads, &fy, &bxy);
                const int zc = std::min(cf.zc, a.nz);
                const int zb = (a.nz + ((a.nz + zc - 1) / zc) - 1) / ((a.nz + zc - 1) / zc);  // balanced
                a.f2_fy = fy;
                a.f2_bxy = bxy;
                a.f2_zchunk = zb;
                b->descs[s].blocks2 = bxy * ((a.nz + zb - 1) / zb);
                smem2 = std::max(smem2, lbm::fused2_smem_bytes(a.nx, fy, b->max_phases));
            }
            prefix[s] = tot;
            prefix2[s] = tot2;
            order[s] = s;
            tot += b->descs[s].blocks;
            tot2 += b->descs[s].blocks2;
        }
        prefix[n_solves] = tot;
        prefix2[n_solves] = tot2;
        b->max_blocks = tot;
        b->max_blocks2 = tot2;
        b->f2_smem = smem2;
        if (b->fused) {
            const int dyn = (int)smem2;
            BCUDA(b, cudaFuncSetAttribute(batch_fused2_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
            BCUDA(b, cudaFuncSetAttribute(batch_fused2_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
        }
        BatchCtl bc{};
        bc.n_active = n_solves;
        bc.total_blocks = tot;
        std::vector<StepArgs> args((size_t)kVariants * n_solves);
        for (int s = 0; s < n_solves; ++s) {
            const BatchDesc& d = b->descs[s];
            const int nz = d.a.nz;
            for (int parity = 0; parity < 2; ++parity)
                for (int frame = 0; frame < 3; ++frame) {
                    StepArgs a = d.a;
                    a.src = d.f[parity];
                    a.dst = d.f[parity ^ 1];
                    a.rsrc = frame == 2 ? d.ref + nz : d.ref;      // 0: AA, 1: AB, 2: BB
                    a.rdst = frame == 0 ? d.ref : d.ref + nz;
                    a.ck.rebase = 1;                              // graph intervals
                    a.ck.steps = b->K;
                    a.ck.use_handle = 0;
                    args[(size_t)s * kVariants + parity * 3 + frame] = a;
                }
        }
        BCUDA(b, cudaMemcpyAsync(b->d_args, args.data(), sizeof(StepArgs) * args.size(),
                                 cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(b->d_descs, b->descs.data(), sizeof(BatchDesc) * n_solves,
                                 cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(b->d_prefix, prefix.data(), sizeof(int) * (n_solves + 1),
                                 cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(b->d_prefix2, prefix2.data(), sizeof(int) * (n_solves + 1),
                                 cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * n_solves,
                                 cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaMemcpyAsync(b->d_bctl, &bc, sizeof bc, cudaMemcpyHostToDevice, st));
        BCUDA(b, cudaStreamSynchronize(st));
        return LBM_OK;
    };

    // The autotuner times each candidate on the batch itself: six plain
    // steps (three two-step launches, or six single steps; state buffer 1 is
    // scratch until the first real step writes it).  Candidates: single steps
    // with 128, 256 or 512 threads, and (FP32, fuse on) two-step launches
    // with 256 .. 640 threads per block and z chunks of 8, 16 or 32 planes.
    // opts.fuse = 2 keeps only the two-step candidates when there are any.
    std::vector<Cfg> cands = {{128, 0, 0}, {256, 0, 0}, {512, 0, 0}};
    if (op.fuse && op.storage == LBM_STORE_F32) {
        std::vector<Cfg> two;
        for (int t2 : {256, 320, 384, 512, 640}) {
            size_t sm = 0;
            if (!f2_ok(t2, &sm)) continue;
            for (int zc : {8, 16, 32}) two.push_back({256, t2, zc});
        }
        if (op.fuse == 2 && !two.empty()) cands = two;
        else cands.insert(cands.end(), two.begin(), two.end());
    }
    Cfg best = cands[0];
    float best_ms = INFINITY;
    for (const Cfg& cf : cands) {
        lbm_status s2 = upload(cf);
        if (s2 != LBM_OK) return s2;
        auto run6 = [&]() -> cudaError_t {
            cudaError_t e = cudaSuccess;
            if (b->fused)
                for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_pair(b, 0, r & 1, st);
            else
                for (int r = 0; r < 6 && e == cudaSuccess; ++r) e = launch_step(b, false, 0, 0, 0u, st);
            return e;
        };
        BCUDA(b, run6());                                  // warm-up
        BCUDA(b, cudaEventRecord(b->ev0, st));
        BCUDA(b, run6());
        BCUDA(b, cudaEventRecord(b->ev1, st));
        BCUDA(b, cudaEventSynchronize(b->ev1));
        float ms = 0.f;
        BCUDA(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        if (ms < best_ms) {
            best_ms = ms;
            best = cf;
        }
    }
    lbm_status s3 = upload(best);
    if (s3 != LBM_OK) return s3;

    // one graph: while (any solve active) { K-1 steps; check step; control }
    const int K = b->K;
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess)
        e = cudaStreamBeginCaptureToGraph(b->cap_stream, np.conditional.phGraph_out[0], nullptr,
                                          nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the interval: one single step into frame R_b, plain steps (as
        // two-step launches in an even number of pairs when the autotuner
        // chose them, so the interval ends in the buffer it started from),
        // the check step, then the control kernel
        const int R = K - 2;
        const int pairs = b->fused ? 2 * (R / 4) : 0;
        int parity = 0, k = 0;
        e = launch_step(b, false, parity, 1, (unsigned)k++, b->cap_stream);
        parity ^= 1;
        for (int i = 0; i < pairs && e == cudaSuccess; ++i, k += 2) {
            e = launch_pair(b, parity, i & 1, b->cap_stream);
            parity ^= 1;
        }
        for (; k < K - 1 && e == cudaSuccess; ++k) {
            e = launch_step(b, false, parity, 2, (unsigned)k, b->cap_stream);
            parity ^= 1;
        }
        if (e == cudaSuccess) e = launch_step(b, true, parity, 2, (unsigned)k, b->cap_stream);
        if (e == cudaSuccess) {
            batch_control_kernel<<<1, 32, 0, b->cap_stream>>>(b->d_descs, n_solves, b->d_prefix,
                                                              b->d_prefix2, b->d_order, b->d_bctl, h, 1);
            e = cudaGetLastError();
        }
        cudaGraph_t captured = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &captured);
        if (e == cudaSuccess) e = e2;
    }
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->poisoned = true;
        return bfail(b, LBM_ERR_CUDA, "building the batch graph failed: %s", cudaGetErrorString(e));
    }
    batch_stamp_kernel<<<1, 1, 0, st>>>(b->d_bctl);
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaEventRecord(b->ev0, st));
    e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev1, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    if (e != cudaSuccess) {
        b->poisoned = true;
        return bfail(b, LBM_ERR_CUDA, "batch graph launch failed: %s", cudaGetErrorString(e));
    }
    float ms = 0.f;
    BCUDA(b, cudaEventElapsedTime(&ms, b->ev0, b->ev1));
#ifdef LBM_DEBUG
    {
        unsigned code = 0;
        BCUDA(b, cudaMemcpyFromSymbol(&code, lbm::g_lbm_debug, sizeof code));
        if (code) return bfail(b, LBM_ERR_INTERNAL, "bounds check %u failed in a batched step kernel", code);
    }
#endif
    long long updates = 0;
    int converged = 0;
    for (int s = 0; s < n_solves; ++s) {
        BCUDA(b, cudaMemcpyAsync(&b->h_ctl[s], b->descs[s].a.ck.ctl, sizeof(Ctl),
                                 cudaMemcpyDeviceToHost, st));
    }
    BCUDA(b, cudaStreamSynchronize(st));
    for (int s = 0; s < n_solves; ++s) {
        const Layout& L = b->layouts[s];
        updates += b->h_ctl[s].iter * (long long)L.NX * L.NY * L.NZ;
        if (b->h_ctl[s].status == LBM_OK) ++converged;
    }
    b->solved = true;
    if (info) {
        info->n_solves = n_solves;
        info->n_converged = converged;
        info->total_updates = updates;
        info->elapsed_ms = ms;
        info->block_threads = b->fused ? b->f2_threads : b->threads;
        info->steps_per_launch = b->fused ? 2 : 1;
        info->reserved = 0;
        info->status = converged == n_solves ? LBM_OK : LBM_ERR_NOT_CONVERGED;
    }
    return LBM_OK;
}

lbm_status lbm_batch_result(const lbm_batch* b, int id, lbm_solve_info* info) {
    if (!b || !info) return LBM_ERR_INVALID_ARG;
    if (!b->solved) return LBM_ERR_STATE;
    if (id < 0 || id >= (int)b->cells.size()) return LBM_ERR_INVALID_ARG;
    const Ctl& c = b->h_ctl[id];
    info->iters = c.iter;
    info->k_eff = c.k_eff;
    info->residual_T = c.r_t;
    info->residual_Q = c.r_q;
    info->elapsed_ms = 0.0;
    info->lattice_scale = b->scale[id];
    info->status = c.status;
    info->checks = (int32_t)c.checks;
    return LBM_OK;
}

lbm_status lbm_batch_get_temperature(lbm_batch* b, int id, float* host_out) {
    if (!b || !host_out) return LBM_ERR_INVALID_ARG;
    if (b->poisoned) return LBM_ERR_CUDA;
    if (!b->solved) return bfail(b, LBM_ERR_STATE, "no solve yet");
    if (id < 0 || id >= (int)b->cells.size()) return bfail(b, LBM_ERR_INVALID_ARG, "bad id");
    BCUDA(b, cudaSetDevice(b->device));
    const Layout& L = b->layouts[id];
    const long long N = (long long)L.n[0] * L.n[1] * L.n[2];
    float* d_T = nullptr;
    BCUDA(b, cudaMalloc((void**)&d_T, sizeof(float) * N));
    // K is even: the state is in buffer 0, in frame R_a
    const BatchDesc& d = b->descs[id];
    if (b->fmt == LBM_STORE_BF16)
        lbm::temperature_kernel<1><<<grid_1d(N), 256, 0, b->stream>>>(d.f[0], d.a.pstride, L, d.ref, d_T);
    else if (b->fmt == LBM_STORE_F16)
        lbm::temperature_kernel<2><<<grid_1d(N), 256, 0, b->stream>>>(d.f[0], d.a.pstride, L, d.ref, d_T);
    else
        lbm::temperature_kernel<0><<<grid_1d(N), 256, 0, b->stream>>>(d.f[0], d.a.pstride, L, d.ref, d_T);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d_T, sizeof(float) * N, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(d_T);
    if (e != cudaSuccess) {
        b->poisoned = true;
        return bfail(b, LBM_ERR_CUDA, "%s", cudaGetErrorString(e));
    }
    return LBM_OK;
}

lbm_status lbm_batch_set_initial(lbm_batch* b, int id, const float* t_init) {
    if (!b) return LBM_ERR_INVALID_ARG;
    if (b->poisoned) return bfail(b, LBM_ERR_CUDA, "batch poisoned by an earlier CUDA error");
    if (id < 0 || id >= (int)b->cells.size()) return bfail(b, LBM_ERR_INVALID_ARG, "bad id");
    Cell& c = b->cells[id];
    if (!t_init) {
        c.t_init.clear();
    } else {
        const size_t N = (size_t)c.n[0] * c.n[1] * c.n[2];
        c.t_init.assign(t_init, t_init + N);
    }
    b->solved = false;
    return LBM_OK;
}

lbm_status lbm_batch_get_history(lbm_batch* b, int id, double* host_out, int max_entries, int* n_out) {
    if (!b || !host_out || max_entries < 0) return LBM_ERR_INVALID_ARG;
    if (b->poisoned) return LBM_ERR_CUDA;
    if (!b->solved) return bfail(b, LBM_ERR_STATE, "no solve yet");
    if (id < 0 || id >= (int)b->cells.size()) return bfail(b, LBM_ERR_INVALID_ARG, "bad id");
    BCUDA(b, cudaSetDevice(b->device));
    const lbm::CheckArgs& k = b->descs[id].a.ck;
    std::vector<double> ring(4 * (size_t)kBatchHistCap);
    std::vector<unsigned long long> tr(kBatchHistCap);
    BatchCtl bc{};
    BCUDA(b, cudaMemcpy(ring.data(), k.hist, sizeof(double) * ring.size(), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(tr.data(), k.hist_t, sizeof(unsigned long long) * tr.size(), cudaMemcpyDeviceToHost));
    BCUDA(b, cudaMemcpy(&bc, b->d_bctl, sizeof bc, cudaMemcpyDeviceToHost));
    const long long checks = b->h_ctl[id].checks;
    const long long kept = std::min<long long>(checks, kBatchHistCap);
    const long long n = std::min<long long>(kept, max_entries);
    for (long long i = 0; i < n; ++i) {
        const long long slot = (checks - n + i) % kBatchHistCap;
        std::memcpy(host_out + 5 * i, &ring[4 * (size_t)slot], sizeof(double) * 4);
        host_out[5 * i + 4] = (double)(long long)(tr[slot] - bc.t0) * 1e-6;
    }
    if (n_out) *n_out = (int)n;
    return LBM_OK;
}

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "null batch"; }

void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    free_device(b);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    cudaGetLastError();
    delete b;
}

}  // extern "C"
