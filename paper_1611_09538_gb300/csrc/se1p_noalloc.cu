// se1p_real_space_noalloc: the real-space sum for callers that cannot allocate
// device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// real-space sum: code running inside a CUDA-graph-building framework whose
// allocator must not be bypassed, embedded hosts whose device memory is
// handed out up front, or plugins loaded into a process that forbids new
// allocations after start-up.  For them this entry point takes the problem
// parameters directly (no plan, whose creation allocates) and keeps all of
// its scratch in one file-scope __device__ array of fixed size.  The array
// exists on every GPU that loads the library, for as long as the process runs.
//
// Limits: at most kNaMaxParticles particles and kNaMaxCells cells per call.
// Every call shares the array and leaves the last call's contents in it;
// calls whose work overlaps on the GPU (different streams, or different host
// threads on the same device) race on it and must be serialised by the caller.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "se1p_plan.h"

using namespace se1p;

namespace {

constexpr int kNaMaxParticles = 16384;
constexpr int kNaMaxCells = 4096;
constexpr int kNaMaxDevices = 64;

// Scratch layout (bytes, each region 256-byte aligned):
//   xyzq    double4 [kNaMaxParticles]       sanitised positions and charges
//   key     int     [kNaMaxParticles]       cell of each particle
//   cells   CellRec<double> [kNaMaxParticles] particles in cell order (also holds the FP32 records)
//   counts  int     [kNaMaxCells]
//   starts  int     [kNaMaxCells + 2]        starts[0] is padding, cell starts from starts[1]
//   cursor  int     [kNaMaxCells]
//   rsum    double  [4][kNaMaxParticles]     real-space sums in cell order
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffXyzq = 0;
constexpr size_t kOffKey = kOffXyzq + align256(sizeof(double) * 4 * kNaMaxParticles);
constexpr size_t kOffCells = kOffKey + align256(sizeof(int) * kNaMaxParticles);
constexpr size_t kOffCounts = kOffCells + align256(sizeof(CellRec<double>) * kNaMaxParticles);
constexpr size_t kOffStarts = kOffCounts + align256(sizeof(int) * kNaMaxCells);
constexpr size_t kOffCursor = kOffStarts + align256(sizeof(int) * (kNaMaxCells + 2));
constexpr size_t kOffRsum = kOffCursor + align256(sizeof(int) * kNaMaxCells);
constexpr size_t kScratchBytes = kOffRsum + align256(sizeof(double) * 4 * kNaMaxParticles);

static __device__ __align__(256) unsigned char g_na_scratch[kScratchBytes];

// Device address of g_na_scratch on each device.  It is looked up again on every call made outside
// stream capture (after cudaDeviceReset the next context may load the module elsewhere); a call
// during capture uses the address of the last uncaptured call on that device.
void *g_na_ptr[kNaMaxDevices] = {};
std::mutex g_na_mutex;

se1p_status na_scratch(cudaStream_t s, void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        cudaGetLastError();
        return SE1P_ERR_CUDA;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    bool capturing = true;  // if the query itself fails, assume capture and keep the cached address
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess) capturing = cs != cudaStreamCaptureStatusNone;
    else cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!capturing || !g_na_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_na_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return SE1P_ERR_CUDA;
        }
        g_na_ptr[dev] = ptr;
    }
    *out = g_na_ptr[dev];
    return SE1P_OK;
}

__global__ void k_na_pack(Geo g, int n, const double *__restrict__ x, const double *__restrict__ q,
                          double *__restrict__ xyzq, int *__restrict__ key, int *__restrict__ counts)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2], qq = q[i];
    if (!isfinite(px)) px = 0.0;
    if (!isfinite(py)) py = 0.0;
    if (!isfinite(pz)) pz = 0.0;
    if (!isfinite(qq)) qq = 0.0;
    px = fmin(fmax(px, 0.0), g.L[0] * (1.0 - 1e-15));
    py = fmin(fmax(py, 0.0), g.L[1] * (1.0 - 1e-15));
    if (pz < 0.0 || pz >= g.L[2]) {  // periodic image in [0, L3): fmod is exact
        pz = fmod(pz, g.L[2]);
        if (pz < 0.0) pz += g.L[2];
        if (pz >= g.L[2]) pz = 0.0;
    }
    const int cx = min((int)(px / g.cs[0]), g.ncx - 1);
    const int cy = min((int)(py / g.cs[1]), g.ncy - 1);
    const int cz = min((int)(pz / g.cs[2]), g.ncz - 1);
    const int cell = (cz * g.ncy + cy) * g.ncx + cx;
    reinterpret_cast<double4 *>(xyzq)[i] = make_double4(px, py, pz, qq);
    key[i] = cell;
    atomicAdd(counts + cell, 1);
}

// Single-block exclusive scan of the cell counts into starts and cursors.
__global__ void k_na_scan(int len, const int *__restrict__ counts, int *__restrict__ starts,
                          int *__restrict__ cursor)
{
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < len; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < len ? counts[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < blockDim.x; o <<= 1) {
            const int t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        const int excl = carry + part[threadIdx.x] - v;
        if (i < len) {
            starts[i] = excl;
            cursor[i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) starts[len] = carry;
}

template <typename T>
__global__ void k_na_scatter(Geo g, int n, const double *__restrict__ xyzq, const int *__restrict__ key,
                             int *__restrict__ cursor, CellRec<T> *__restrict__ cells)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4_32a p = reinterpret_cast<const double4_32a *>(xyzq)[i];  // 32-byte records
    const int cell = key[i];
    const int pos = atomicAdd(cursor + cell, 1);
    CellRec<T> c;
    c.xh = (T)p.x;
    c.yh = (T)p.y;
    c.zh = (T)p.z;
    c.xl = (T)(p.x - (double)c.xh);
    c.yl = (T)(p.y - (double)c.yh);
    c.zl = (T)(p.z - (double)c.zh);
    c.q = (T)p.w;
    c.orig = i;
    cells[pos] = c;
}

template <typename T>
se1p_status na_run(const se1p_params &P, const Geo &g, unsigned char *scr, int n, const double *x, const double *q,
                   double *phi, double *force, cudaStream_t s)
{
    double *xyzq = reinterpret_cast<double *>(scr + kOffXyzq);
    int *key = reinterpret_cast<int *>(scr + kOffKey);
    CellRec<T> *cells = reinterpret_cast<CellRec<T> *>(scr + kOffCells);
    int *counts = reinterpret_cast<int *>(scr + kOffCounts);
    int *starts = reinterpret_cast<int *>(scr + kOffStarts);
    int *cursor = reinterpret_cast<int *>(scr + kOffCursor);
    double *rsum = reinterpret_cast<double *>(scr + kOffRsum);
    // counts must start at zero on every call (the array keeps the previous call's values)
    if (cudaMemsetAsync(counts, 0, sizeof(int) * g.ncells, s) != cudaSuccess) return SE1P_ERR_CUDA;
    const int bs = 256, nb = (n + bs - 1) / bs;
    k_na_pack<<<nb, bs, 0, s>>>(g, n, x, q, xyzq, key, counts);
    k_na_scan<<<1, 1024, 0, s>>>(g.ncells, counts, starts + 1, cursor);
    k_na_scatter<T><<<nb, bs, 0, s>>>(g, n, xyzq, key, cursor, cells);
    // The real-space kernel reads a plan's buffers; describe the scratch regions
    // with a plan object on the host stack (nothing is allocated).
    se1p_plan view;
    view.prm = P;
    view.geo = g;
    view.b.starts = starts;  // cell starts begin at starts + nbins + 1 = starts + 1
    view.b.cells = cells;
    view.b.rsum = rsum;
    launch_real_space<T>(&view, n, key, phi, force, 0, s);
    return cudaGetLastError() == cudaSuccess ? SE1P_OK : SE1P_ERR_CUDA;
}

}  // namespace

extern "C" se1p_status se1p_real_space_noalloc(const se1p_params *params, int n, const double *x,
                                               const double *q, double *phi, double *force, void *stream)
{
    if (!params || n < 0 || (n > 0 && (!x || !q || !phi || !force))) return SE1P_ERR_INVALID_ARG;
    const se1p_params &P = *params;
    for (int i = 0; i < 3; ++i)
        if (!(P.L[i] > 0.0) || !isfinite(P.L[i])) return SE1P_ERR_INVALID_ARG;
    if (!(P.xi > 0.0) || !isfinite(P.xi) || !(P.rc > 0.0) || !isfinite(P.rc) || P.rc > P.L[2])
        return SE1P_ERR_INVALID_ARG;
    if (P.precision != SE1P_FP64 && P.precision != SE1P_MIXED) return SE1P_ERR_INVALID_ARG;
    if (n > kNaMaxParticles) return SE1P_ERR_CAPACITY;
    if (n == 0) return SE1P_OK;

    Geo g{};
    for (int i = 0; i < 3; ++i) g.L[i] = P.L[i];
    g.xi = P.xi;
    g.rc = P.rc;
    g.rc2 = P.rc * P.rc;
    // cells no smaller than rc, at most kNaMaxCells of them (coarser cells stay >= rc)
    int nc[3];
    for (int i = 0; i < 3; ++i) nc[i] = (int)fmin(fmax(floor(P.L[i] / P.rc), 1.0), 4096.0);
    while ((long)nc[0] * nc[1] * nc[2] > kNaMaxCells) {
        int a = 0;
        for (int i = 1; i < 3; ++i)
            if (nc[i] > nc[a]) a = i;
        nc[a] = (nc[a] + 1) / 2;
    }
    g.ncx = nc[0];
    g.ncy = nc[1];
    g.ncz = nc[2];
    g.ncells = nc[0] * nc[1] * nc[2];
    for (int i = 0; i < 3; ++i) g.cs[i] = P.L[i] / nc[i];
    g.nbins = 0;

    cudaStream_t s = (cudaStream_t)stream;
    void *scr = nullptr;
    se1p_status st = na_scratch(s, &scr);
    if (st != SE1P_OK) return st;
    return P.precision == SE1P_MIXED
               ? na_run<float>(P, g, (unsigned char *)scr, n, x, q, phi, force, s)
               : na_run<double>(P, g, (unsigned char *)scr, n, x, q, phi, force, s);
}
