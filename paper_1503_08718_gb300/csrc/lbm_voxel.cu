// Device voxeliser of the synthetic four-directional braided unit cell.
//
// Step-wise approximation of curved yarn boundaries (Section 3.2): a voxel
// belongs to a yarn when its centre lies inside the yarn's elliptic section.
// Yarns run at the interior braiding angle g from z (Section 4.1) in four
// families.  Every FP64 operation of the membership test is an explicitly
// rounded intrinsic evaluated left to right, with no fused multiply-add, so
// the phase map is reproducible bit for bit by any implementation that
// follows the same recipe; the host part is compiled without contraction.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "lbm.h"

extern "C" {
uint8_t* lbm__device_phase(lbm_ctx* c);
int lbm__dims(const lbm_ctx* c, int* n);
void lbm__set_phase_count(lbm_ctx* c, int n_phases);
void lbm__set_error(lbm_ctx* c, const char* msg);
int lbm__poisoned(const lbm_ctx* c);
void lbm__poison(lbm_ctx* c);
int lbm__voxel_scratch(lbm_ctx* c, int n_max, double2** anchors, unsigned long long** hist);
}

namespace {

constexpr int kMaxYarns = 4096;

struct Braid {
    double d[4][3], u[4][3], v[4][3];   // axis, horizontal major direction, minor direction
    double A, B, Nx, Ny;
    int nx, ny, nz;
};

// Voxel-centre test for one yarn; the order of operations is part of the
// recipe (see the file comment).
__device__ __forceinline__ bool inside(const Braid& b, int fam, double x0, double y0, double cx,
                                       double cy, double cz) {
    const double* d = b.d[fam];
    const double* u = b.u[fam];
    const double* v = b.v[fam];
    const double t = __ddiv_rn(cz, d[2]);
    const double px = __dadd_rn(x0, __dmul_rn(d[0], t));
    const double py = __dadd_rn(y0, __dmul_rn(d[1], t));
    double rx = __dsub_rn(cx, px);
    double ry = __dsub_rn(cy, py);
    rx = __dsub_rn(rx, __dmul_rn(b.Nx, floor(__dadd_rn(__ddiv_rn(rx, b.Nx), 0.5))));
    ry = __dsub_rn(ry, __dmul_rn(b.Ny, floor(__dadd_rn(__ddiv_rn(ry, b.Ny), 0.5))));
    const double rd = __dadd_rn(__dmul_rn(rx, d[0]), __dmul_rn(ry, d[1]));
    const double wx = __dsub_rn(rx, __dmul_rn(rd, d[0]));
    const double wy = __dsub_rn(ry, __dmul_rn(rd, d[1]));
    const double wz = -__dmul_rn(rd, d[2]);
    const double a = __ddiv_rn(__dadd_rn(__dmul_rn(wx, u[0]), __dmul_rn(wy, u[1])), b.A);
    const double bb = __ddiv_rn(
        __dadd_rn(__dadd_rn(__dmul_rn(wx, v[0]), __dmul_rn(wy, v[1])), __dmul_rn(wz, v[2])), b.B);
    return __dadd_rn(__dmul_rn(a, a), __dmul_rn(bb, bb)) <= 1.0;
}

__device__ __forceinline__ int first_yarn(const Braid& b, const double2* __restrict__ anchors,
                                          int n, long long vox) {
    const int x = (int)(vox % b.nx);
    const long long r = vox / b.nx;
    const int y = (int)(r % b.ny);
    const int z = (int)(r / b.ny);
    const double cx = (double)x + 0.5, cy = (double)y + 0.5, cz = (double)z + 0.5;
    for (int i = 0; i < n; ++i) {
        const double2 p = anchors[i];
        if (inside(b, i & 3, p.x, p.y, cx, cy, cz)) return i;
    }
    return n;
}

// Histogram of the first containing yarn over all voxels (bin n_max = none).
__global__ void braid_count_kernel(Braid b, const double2* __restrict__ anchors, int n_max,
                                   unsigned long long* __restrict__ hist) {
    extern __shared__ unsigned int s_hist[];
    for (int i = threadIdx.x; i <= n_max; i += blockDim.x) s_hist[i] = 0u;
    __syncthreads();
    const long long N = (long long)b.nx * b.ny * b.nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x)
        atomicAdd(&s_hist[first_yarn(b, anchors, n_max, v)], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i <= n_max; i += blockDim.x)
        if (s_hist[i]) atomicAdd(&hist[i], (unsigned long long)s_hist[i]);
}

__global__ void braid_write_kernel(Braid b, const double2* __restrict__ anchors, int n_used,
                                   uint8_t* __restrict__ phase) {
    const long long N = (long long)b.nx * b.ny * b.nz;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < N;
         v += (long long)gridDim.x * blockDim.x) {
        const int f = first_yarn(b, anchors, n_used, v);
        phase[v] = f < n_used ? (uint8_t)(1 + (f & 3)) : (uint8_t)0;
    }
}

}  // namespace

extern "C" lbm_status lbm_set_geometry_braid(lbm_ctx* c, double g_rad, double A, double B,
                                             const double* anchors, int n_max, double phi,
                                             int* n_used, double* fraction) {
    if (!c) return LBM_ERR_INVALID_ARG;
    if (lbm__poisoned(c)) return LBM_ERR_CUDA;
    if (!anchors || n_max < 1 || n_max > kMaxYarns || !(A > 0.0) || !(B > 0.0) ||
        !(g_rad > 0.0) || !(g_rad < 1.5707963267948966) || !(phi >= 0.0) || !(phi <= 1.0)) {
        lbm__set_error(c, "invalid braid parameters (need 0 < g < pi/2, A, B > 0, 1 <= n_max <= 4096, 0 <= phi <= 1)");
        return LBM_ERR_INVALID_ARG;
    }
    int n[3];
    const int dev = lbm__dims(c, n);
    Braid b;
    static const int SX[4] = {1, -1, -1, 1};
    static const int SY[4] = {1, 1, -1, -1};
    const double h = std::sin(g_rad) / std::sqrt(2.0);
    const double cg = std::cos(g_rad);
    for (int k = 0; k < 4; ++k) {
        double* d = b.d[k];
        double* u = b.u[k];
        double* v = b.v[k];
        d[0] = SX[k] * h;
        d[1] = SY[k] * h;
        d[2] = cg;
        const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1]);
        u[0] = -d[1] / nrm;
        u[1] = d[0] / nrm;
        u[2] = 0.0;
        v[0] = -(d[2] * u[1]);
        v[1] = d[2] * u[0];
        v[2] = d[0] * u[1] - d[1] * u[0];
    }
    b.A = A;
    b.B = B;
    b.Nx = (double)n[0];
    b.Ny = (double)n[1];
    b.nx = n[0];
    b.ny = n[1];
    b.nz = n[2];
    const long long N = (long long)n[0] * n[1] * n[2];

    double2* d_anchor = nullptr;
    unsigned long long* d_hist = nullptr;
    std::vector<unsigned long long> hist((size_t)n_max + 1, 0ull);
    cudaError_t e = cudaSetDevice(dev);
    // a context on a caller's workspace keeps this scratch inside it
    const bool own = !lbm__voxel_scratch(c, n_max, &d_anchor, &d_hist);
    if (e == cudaSuccess && own) e = cudaMalloc((void**)&d_anchor, sizeof(double2) * n_max);
    if (e == cudaSuccess && own) e = cudaMalloc((void**)&d_hist, sizeof(unsigned long long) * (n_max + 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_anchor, anchors, sizeof(double2) * n_max, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d_hist, 0, sizeof(unsigned long long) * (n_max + 1));
    long long blocks = (N + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (e == cudaSuccess) {
        braid_count_kernel<<<(int)blocks, 256, sizeof(unsigned int) * (n_max + 1)>>>(b, d_anchor, n_max,
                                                                                     d_hist);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(hist.data(), d_hist, sizeof(unsigned long long) * (n_max + 1), cudaMemcpyDeviceToHost);
    int used = -1;
    unsigned long long cum = 0;
    if (e == cudaSuccess) {
        for (int i = 0; i < n_max; ++i) {
            cum += hist[i];
            if ((double)cum >= phi * (double)N) {
                used = i + 1;
                break;
            }
        }
    }
    if (e == cudaSuccess && used > 0) {
        braid_write_kernel<<<(int)blocks, 256>>>(b, d_anchor, used, lbm__device_phase(c));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (own) {
        cudaFree(d_anchor);
        cudaFree(d_hist);
    }
    if (e != cudaSuccess) {
        lbm__poison(c);
        lbm__set_error(c, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (used < 0) {
        lbm__set_error(c, "yarn fraction phi not reached with n_max yarns");
        return LBM_ERR_INVALID_ARG;
    }
    unsigned long long yarn = 0;
    for (int i = 0; i < used; ++i) yarn += hist[i];
    if (n_used) *n_used = used;
    if (fraction) *fraction = (double)yarn / (double)N;
    lbm__set_phase_count(c, 5);
    return LBM_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the braided-cell voxeliser.
//
// Some callers cannot call cudaMalloc: a process whose device memory is owned
// by another allocator (for instance a deep-learning framework's caching
// pool that has reserved most of the GPU), a service running under a fixed
// memory budget, or a latency-sensitive loop that must not stall on the
// implicit device synchronisation of cudaMalloc / cudaFree.  For them the
// histogram that the voxeliser needs as scratch lives in a file-scope device
// array of fixed size instead of a per-call allocation; inputs and outputs
// stay in the caller's memory.
// ---------------------------------------------------------------------------

namespace {

constexpr int kNoAllocMaxYarns = LBM_NOALLOC_MAX_YARNS;
constexpr int kMaxDevices = 64;

// Scratch histogram: one bin per yarn plus the "no yarn" bin.  Every device
// that loads the library holds this array until the process exits.  All
// calls on a device share it.
static __device__ __align__(256) unsigned long long g_noalloc_hist[kNoAllocMaxYarns + 1];

// Device address of g_noalloc_hist per device, looked up once per device
// (by the first call on it).  The address holds for the life of the device's
// primary context: a process that resets the device (cudaDeviceReset) must
// not call this entry point again.
unsigned long long* g_hist_addr[kMaxDevices] = {};
std::mutex g_hist_mutex;

void put_msg(char* err, int err_len, const char* msg) {
    if (err && err_len > 0) {
        std::strncpy(err, msg, (size_t)err_len - 1);
        err[err_len - 1] = '\0';
    }
}

}  // namespace

extern "C" lbm_status lbm_braid_voxelize_noalloc(int nx, int ny, int nz, double g_rad, double A,
                                                 double B, const double* d_anchors, int n_max,
                                                 double phi, uint8_t* d_phase, int* n_used,
                                                 double* fraction, void* stream, char* err,
                                                 int err_len) {
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz >= (1LL << 31)) {
        put_msg(err, err_len, "cell sizes must be >= 1 with nx*ny*nz < 2^31");
        return LBM_ERR_INVALID_ARG;
    }
    if (n_max < 1 || n_max > kNoAllocMaxYarns) {
        put_msg(err, err_len, "n_max must be in [1, LBM_NOALLOC_MAX_YARNS = 1024]: the scratch "
                              "histogram of the allocation-free voxeliser has 1025 bins");
        return LBM_ERR_INVALID_ARG;
    }
    if (!d_anchors || !d_phase || ((uintptr_t)d_anchors & 15u)) {
        put_msg(err, err_len, "d_anchors (16-byte aligned) and d_phase must be device pointers");
        return LBM_ERR_INVALID_ARG;
    }
    if (!(A > 0.0) || !(B > 0.0) || !(g_rad > 0.0) || !(g_rad < 1.5707963267948966) ||
        !(phi >= 0.0) || !(phi <= 1.0)) {
        put_msg(err, err_len, "need 0 < g < pi/2, A > 0, B > 0 and 0 <= phi <= 1");
        return LBM_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        put_msg(err, err_len, e != cudaSuccess ? cudaGetErrorString(e) : "device index too large");
        return LBM_ERR_CUDA;
    }
    // both buffers must be memory this device can address: a host pointer
    // passed by mistake would otherwise fault inside the kernels
    {
        const void* ptrs[2] = {d_anchors, d_phase};
        for (const void* p : ptrs) {
            cudaPointerAttributes pa;
            const cudaError_t ea = cudaPointerGetAttributes(&pa, p);
            if (ea != cudaSuccess || !(pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged) ||
                (pa.type == cudaMemoryTypeDevice && pa.device != dev)) {
                cudaGetLastError();
                put_msg(err, err_len, "d_anchors and d_phase must be device (or managed) memory of the "
                                      "current device");
                return LBM_ERR_INVALID_ARG;
            }
        }
    }
    unsigned long long* hist = nullptr;
    {
        // set-up on the first call on this device (the current device)
        std::lock_guard<std::mutex> lock(g_hist_mutex);
        if (!g_hist_addr[dev]) {
            e = cudaGetSymbolAddress((void**)&g_hist_addr[dev], g_noalloc_hist);
            if (e != cudaSuccess) {
                g_hist_addr[dev] = nullptr;
                put_msg(err, err_len, cudaGetErrorString(e));
                return LBM_ERR_CUDA;
            }
        }
        hist = g_hist_addr[dev];
    }

    Braid b;
    static const int SX[4] = {1, -1, -1, 1};
    static const int SY[4] = {1, 1, -1, -1};
    const double h = std::sin(g_rad) / std::sqrt(2.0);
    const double cg = std::cos(g_rad);
    for (int k = 0; k < 4; ++k) {
        double* d = b.d[k];
        double* u = b.u[k];
        double* v = b.v[k];
        d[0] = SX[k] * h;
        d[1] = SY[k] * h;
        d[2] = cg;
        const double nrm = std::sqrt(d[0] * d[0] + d[1] * d[1]);
        u[0] = -d[1] / nrm;
        u[1] = d[0] / nrm;
        u[2] = 0.0;
        v[0] = -(d[2] * u[1]);
        v[1] = d[2] * u[0];
        v[2] = d[0] * u[1] - d[1] * u[0];
    }
    b.A = A;
    b.B = B;
    b.Nx = (double)nx;
    b.Ny = (double)ny;
    b.nx = nx;
    b.ny = ny;
    b.nz = nz;
    const long long N = (long long)nx * ny * nz;
    cudaStream_t st = (cudaStream_t)stream;
    const double2* anchors = reinterpret_cast<const double2*>(d_anchors);

    // the array keeps the previous call's counts: clear the bins this call uses
    const size_t bytes = sizeof(unsigned long long) * ((size_t)n_max + 1);
    e = cudaMemsetAsync(hist, 0, bytes, st);
    long long blocks = (N + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    if (e == cudaSuccess) {
        braid_count_kernel<<<(int)blocks, 256, sizeof(unsigned int) * (n_max + 1), st>>>(
            b, anchors, n_max, hist);
        e = cudaGetLastError();
    }
    unsigned long long counts[kNoAllocMaxYarns + 1];
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, hist, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        put_msg(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    int used = -1;
    unsigned long long cum = 0;
    for (int i = 0; i < n_max; ++i) {
        cum += counts[i];
        if ((double)cum >= phi * (double)N) {
            used = i + 1;
            break;
        }
    }
    if (used < 0) {
        put_msg(err, err_len, "yarn fraction phi not reached with n_max yarns");
        return LBM_ERR_INVALID_ARG;
    }
    braid_write_kernel<<<(int)blocks, 256, 0, st>>>(b, anchors, used, d_phase);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        put_msg(err, err_len, cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    if (n_used) *n_used = used;
    if (fraction) *fraction = (double)cum / (double)N;
    put_msg(err, err_len, "");
    return LBM_OK;
}
