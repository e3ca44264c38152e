// Particle-side kernels of the SE1P path:
//   pack + validate -> counting sort into spread bins and real-space cells,
//   per-particle Gaussian window tables, gridding (Eq. 3.4), gathering
//   (Eq. 3.11) with its analytic gradient (Eq. 3.25), and the final FP64
//   energy reduction U = 1/2 sum q phi.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "se1p_plan.h"

namespace se1p {

namespace {

__device__ __forceinline__ int support_start(double t, int P)
{
    // even P: floor(t) - P/2 + 1 ... floor(t) + P/2; odd P: centred on round(t)
    return (P & 1) ? (int)floor(t + 0.5) - (P - 1) / 2 : (int)floor(t) - P / 2 + 1;
}

__device__ __forceinline__ int imod(int a, int m)
{
    int r = a % m;
    return r < 0 ? r + m : r;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Free-axis and z support starts of a sanitised particle.
// Grid coordinate t = x / h.  The product x (1/h) is within a few ulps of the correctly
// rounded quotient; it can only change the support start (floor(t) for even P, floor(t + 1/2)
// for odd P) when t lies that close to an integer (even P) or a half-integer (odd P), e.g. a
// charge on a grid node.  There the quotient is taken exactly, so that the support is the one
// the plain definition gives (FP64 division is slow on this part, and almost never needed).
__device__ __forceinline__ double grid_coord(double xs, double h, double inv_h, int P)
{
    double t = xs * inv_h;
    const double b = (P & 1) ? floor(t) + 0.5 : rint(t);  // nearest decision boundary
    if (fabs(t - b) <= 1e-14 * fmax(fabs(t), 1.0)) t = xs / h;
    return t;
}

// Periodic image in [0, L): fmod is exact.
__device__ __forceinline__ double wrap_periodic(double v, double L)
{
    if (v < 0.0 || v >= L) {
        v = fmod(v, L);
        if (v < 0.0) v += L;
        if (v >= L) v = 0.0;
    }
    return v;
}

struct Support {
    int i0[3];
    double t[3];
};

__device__ __forceinline__ Support particle_support(const Geo &g, double px, double py, double pz)
{
    Support s;
    s.t[0] = grid_coord(px + g.off, g.h, g.inv_h, g.P);
    s.t[1] = grid_coord(py + g.off, g.h, g.inv_h, g.P);
    s.t[2] = grid_coord(pz, g.hz, g.inv_hz, g.P);
    const int hi = g.Mt - g.P;
    s.i0[0] = min(max(support_start(s.t[0], g.P), 0), hi);
    s.i0[1] = min(max(support_start(s.t[1], g.P), 0), hi);
    s.i0[2] = support_start(s.t[2], g.P);  // unwrapped
    return s;
}

// ------------------------------------------------------------------ pack
template <typename T>
__global__ void k_pack(Geo g, int n, const double *__restrict__ x, const double *__restrict__ q,
                       double *__restrict__ xyzq, int *__restrict__ bin_key, int *__restrict__ cell_key,
                       int *__restrict__ bin_count, int *__restrict__ cell_count, double *__restrict__ sums,
                       int *__restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double sq = 0.0, saq = 0.0;
    if (i < n) {
        double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2], qq = q[i];
        int flag = 0;
        if (!isfinite(px) || !isfinite(py) || !isfinite(pz) || !isfinite(qq)) {
            flag |= FLAG_NAN;
            if (!isfinite(px)) px = 0.0;
            if (!isfinite(py)) py = 0.0;
            if (!isfinite(pz)) pz = 0.0;
            qq = 0.0;
        }
        if (g.per3) {  // triply periodic: x and y are wrapped like z
            px = wrap_periodic(px, g.L[0]);
            py = wrap_periodic(py, g.L[1]);
        } else if (px < 0.0 || px >= g.L[0] || py < 0.0 || py >= g.L[1]) {
            flag |= FLAG_OUT_OF_BOX;
            px = fmin(fmax(px, 0.0), g.L[0] * (1.0 - 1e-15));
            py = fmin(fmax(py, 0.0), g.L[1] * (1.0 - 1e-15));
        }
        pz = wrap_periodic(pz, g.L[2]);
        const Support s = particle_support(g, px, py, pz);
        const int bx = s.i0[0] / kBin, by = s.i0[1] / kBin, bz = imod(s.i0[2], g.M3) / kBin;
        const int bin = (bz * g.nby + by) * g.nbx + bx;
        const int cx = min((int)(px / g.cs[0]), g.ncx - 1);
        const int cy = min((int)(py / g.cs[1]), g.ncy - 1);
        const int cz = min((int)(pz / g.cs[2]), g.ncz - 1);
        const int cell = (cz * g.ncy + cy) * g.ncx + cx;
        reinterpret_cast<double4 *>(xyzq)[i] = make_double4(px, py, pz, qq);
        bin_key[i] = bin;
        cell_key[i] = cell;
        atomicAdd(bin_count + bin, 1);
        atomicAdd(cell_count + cell, 1);
        if (flag) atomicOr(status, flag);
        sq = qq;
        saq = fabs(qq);
    }
    // the CTA's charge sums, then one pair of atomic adds per CTA (per warp, the two addresses
    // received thousands of same-address atomics per evaluation)
    __shared__ double ws[2][32];
    sq = warp_sum(sq);
    saq = warp_sum(saq);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        ws[0][w] = sq;
        ws[1][w] = saq;
    }
    __syncthreads();
    if (w == 0) {
        sq = lane < nw ? ws[0][lane] : 0.0;
        saq = lane < nw ? ws[1][lane] : 0.0;
        sq = warp_sum(sq);
        saq = warp_sum(saq);
        if (lane == 0 && (sq != 0.0 || saq != 0.0)) {
            atomicAdd(sums, sq);
            atomicAdd(sums + 1, saq);
        }
    }
}

// Exclusive scans of the bin and cell histograms (one block per array); the
// first block also checks neutrality, |sum q| <= 1e-12 sum |q| (Section 2.1).
__global__ void k_scan(int nbins, int ncells, const int *__restrict__ counts, int *__restrict__ starts,
                       int *__restrict__ cursors, const double *__restrict__ sums, int *__restrict__ status,
                       int check_neutral)
{
    const int which = blockIdx.x;
    const int len = which == 0 ? nbins : ncells;
    const int *c = counts + (which == 0 ? 0 : nbins);
    int *st = starts + (which == 0 ? 0 : nbins + 1);
    int *cu = cursors + (which == 0 ? 0 : nbins);
    __shared__ int warp_tot[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int base = 0; base < len; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = i < len ? c[i] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = lane < nw ? warp_tot[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            if (lane < nw) warp_tot[lane] = wi - w;  // exclusive warp offsets
        }
        __syncthreads();
        const int excl = carry + warp_tot[wid] + incl - v;
        if (i < len) {
            st[i] = excl;
            cu[i] = excl;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) st[len] = carry;
    if (which == 0 && threadIdx.x == 0 && check_neutral) {
        if (fabs(sums[0]) > 1e-12 * sums[1]) atomicOr(status, FLAG_NOT_NEUTRAL);
    }
}

// Multi-block exclusive scan of the cell counts (used when there are many cells): per-block
// sums, one block scanning those into block offsets, then each block rescanning its chunk.
constexpr int kScanThreads = 256, kScanItems = kScanChunk / kScanThreads;

// Exclusive scan of one value per thread over the block (kScanThreads threads); every thread
// also receives the block's total.
__device__ __forceinline__ int block_exclusive_scan(int v, int &total)
{
    constexpr int NW = kScanThreads / 32;
    __shared__ int wsum[NW + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < NW ? wsum[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < NW) wsum[lane] = wi - w;  // exclusive warp offsets
        if (lane == NW - 1) wsum[NW] = wi;   // block total
    }
    __syncthreads();
    const int r = wsum[wid] + incl - v;
    total = wsum[NW];
    __syncthreads();  // wsum is reused by the next call
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int len, const int *__restrict__ c, int *__restrict__ bsum)
{
    const int base = blockIdx.x * kScanChunk;
    int s = 0;
    for (int k = threadIdx.x; k < kScanChunk; k += kScanThreads)
        if (base + k < len) s += c[base + k];
    int total;
    block_exclusive_scan(s, total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_offsets(int nblk, int *__restrict__ bsum)
{
    int carry = 0;
    for (int base = 0; base < nblk; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const int v = i < nblk ? bsum[i] : 0;
        int total;
        const int e = block_exclusive_scan(v, total);
        if (i < nblk) bsum[i] = carry + e;
        carry += total;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_write(int len, const int *__restrict__ c,
                                                              const int *__restrict__ boff, int *__restrict__ st,
                                                              int *__restrict__ cu)
{
    const int base = blockIdx.x * kScanChunk + threadIdx.x * kScanItems;
    int v[kScanItems];
    int ts = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < len ? c[base + k] : 0;
        ts += v[k];
    }
    int total;
    int e = boff[blockIdx.x] + block_exclusive_scan(ts, total);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < len) {
            st[base + k] = e;
            cu[base + k] = e;
            if (base + k == len - 1) st[len] = e + v[k];
        }
        e += v[k];
    }
}

// Scatter into bin order (with the window tables) and into cell order.  One thread per
// particle computes its window values into a per-warp shared buffer (row stride 3P + 1, so the
// lanes' rows start in different banks); the warp then writes each particle's row of 3P values
// to the table with consecutive lanes on consecutive elements.
constexpr int kScatterThreads = 64;  // FP64 launches half of it: its buffer stays below 48 KB

template <typename T>
__global__ void __launch_bounds__(kScatterThreads) k_scatter(Geo g, int n, const double *__restrict__ xyzq,
                                                             const int *__restrict__ bin_key,
                                                             const int *__restrict__ cell_key,
                                                             int *__restrict__ bin_cursor,
                                                             int *__restrict__ cell_cursor,
                                                             PartRec<T> *__restrict__ parts,
                                                             T *__restrict__ wts, CellRec<T> *__restrict__ cells)
{
    extern __shared__ __align__(16) unsigned char scatter_raw[];
    const int rowlen = 3 * g.P, rs = rowlen + 1;
    const int lane = threadIdx.x & 31;
    T *stage = reinterpret_cast<T *>(scatter_raw) + (threadIdx.x >> 5) * 32 * rs;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int pos = -1;
    if (i < n) {
        const double4_32a p = reinterpret_cast<const double4_32a *>(xyzq)[i];  // 32-byte records
        const Support s = particle_support(g, p.x, p.y, p.z);
        pos = atomicAdd(bin_cursor + bin_key[i], 1);
        PartRec<T> r;
        r.i0[0] = s.i0[0];
        r.i0[1] = s.i0[1];
        r.i0[2] = imod(s.i0[2], g.M3);
        r.orig = i;
        r.q = (T)p.w;
        T *w = stage + lane * rs;
        // Unnormalised windows exp(-alpha d^2): the normalisation (2 xi^2 / (pi eta))^{1/2}
        // per axis is applied once, in FP64, after the gather, so that no rounded constant
        // biases the FP32 grid (a bias there would not cancel against the self term).
        for (int a = 0; a < 3; ++a) {
            const double gg = s.t[a] - s.i0[a] - g.c;  // particle offset from the support centre, grid units
            r.g[a] = (T)gg;
            const double alpha = a < 2 ? g.alpha_xy : g.alpha_z;
            if constexpr (sizeof(T) == sizeof(double)) {
                for (int j = 0; j < g.P; ++j) {
                    const double d = gg - (double)(j - g.c);
                    w[a * g.P + j] = exp(-alpha * d * d);
                }
            } else {
                // FP32 window: |gg| < 1, so gg - (j - c) is exact to ~6e-8 absolute; alpha is
                // split into hi + lo so that its rounding does not bias every exponent alike
                const float gf = (float)gg, ah = (float)alpha, al = (float)(alpha - (double)ah);
                for (int j = 0; j < g.P; ++j) {
                    const float d = gf - (float)(j - g.c);
                    const float d2 = d * d;
                    w[a * g.P + j] = exp_window(-fmaf(ah, d2, al * d2));
                }
            }
        }
        parts[pos] = r;
        // cell order, absolute coordinates as hi + lo
        const int cell = cell_key[i];
        const int cpos = atomicAdd(cell_cursor + cell, 1);
        CellRec<T> c;
        c.xh = (T)p.x;
        c.yh = (T)p.y;
        c.zh = (T)p.z;
        c.xl = (T)(p.x - (double)c.xh);
        c.yl = (T)(p.y - (double)c.yh);
        c.zl = (T)(p.z - (double)c.zh);
        c.q = (T)p.w;
        c.orig = i;
        cells[cpos] = c;
    }
    __syncwarp();
    for (int k = 0; k < 32; ++k) {
        const int pk = __shfl_sync(0xffffffffu, pos, k);
        if (pk < 0) continue;  // warp-uniform
        T *dst = wts + (size_t)pk * rowlen;
        const T *src = stage + k * rs;
        for (int e = lane; e < rowlen; e += 32) dst[e] = src[e];
    }
}

// ------------------------------------------------------------------ gridding (Eq. 3.4)
//
// Output-stationary: a CTA owns an 8x8x8 tile of the grid and accumulates in
// registers every particle whose support overlaps it; kSpreadSplit CTAs may share
// a tile (alternate z bins) and add their partial tiles into the zeroed grid, one
// atomic add per grid point each.  A 16-thread group covers the tile with
// 2(z) x 2(y) x 8(x) points per thread, so each particle costs a thread 4
// shared loads (its z, y and x window values) for 32 FMAs; the CTA's eight
// groups take alternate particles and their partial tiles are added at the end.
// The tile's particles are those of the bins (8 support-start indices per axis)
// whose supports can reach it: a few (z, y) rows of bins, each one contiguous
// range of the bin-sorted records; the ranges are loaded together and taken as one
// list in full batches (batches per row left many partial ones where tiles hold few
// particles).
// At the end every group's partial tile goes to shared memory (reusing the batch
// buffers) and all threads sum it, each 4 of the 512 points over the 8 groups
// (one half-warp summing the others' partial tiles made up a large part of the
// time of tiles with few particles: N = 10^6 in [1, 1, 8], 3.57 -> 3.21 ms).
// A batch of 128 records is loaded once into shared memory, then one thread
// per (particle, axis) gathers the window values at the tile's 8 offsets
// (zero outside the support, charge folded into z).
constexpr int kSpreadBatch = 128;
constexpr int kSpreadGroups = 8;
constexpr int kSpreadThreads = 16 * kSpreadGroups;
// CTAs per tile, each taking every kSpreadSplit-th z bin (atomic combine).  Alone, 2 is faster
// (0.44 against 0.58 ms at C2); alongside the concurrent real space, 1 leaves it more of the SMs
// and the evaluation is faster (1.599 against 1.610 ms).
constexpr int kSpreadSplit = 1;
// CTAs per SM the FP32 kernel is compiled for (72 registers): against the compiler's own choice
// (68) and six (80), seven gave the fastest evaluations (N = 10^5: 1.461 ms; N = 10^6 in [1, 1, 8]:
// 11.51 ms; 64 systems: 17.84 ms)
constexpr int kSpreadMinBlocks = 7;
// rows of bins per tile: at most 7 z bins (a cyclic range of P + 7 <= 39 starts, or all of a z axis
// shorter than P + 23) times 6 y bins (P <= 32)
constexpr int kSpreadMaxRows = 64;

template <typename T>
__global__ void __launch_bounds__(kSpreadThreads, sizeof(T) == 4 ? kSpreadMinBlocks : 1) k_spread(Geo g, const int *__restrict__ bin_start,
                                                           const PartRec<T> *__restrict__ parts,
                                                           const T *__restrict__ wts, T *__restrict__ grid)
{
    // the groups' partial tiles for the final sum: [group][r kBin + c][thread], each group's block
    // padded by 16 values so that the two groups of a warp store to different banks; it reuses the
    // batch buffers (window values, offsets, charges)
    constexpr int kRedStride = 4 * kBin * 16 + 16;
    constexpr size_t kSwBytes = sizeof(T) * kSpreadBatch * 3 * kBin, kOffBytes = sizeof(int) * kSpreadBatch * 3;
    constexpr size_t kBatchBytes = kSwBytes + kOffBytes + sizeof(T) * kSpreadBatch;
    constexpr size_t kRedBytes = sizeof(T) * kSpreadGroups * kRedStride;
    __shared__ __align__(16) unsigned char sraw[kBatchBytes > kRedBytes ? kBatchBytes : kRedBytes];
    T(*sw)[3][kBin] = reinterpret_cast<T(*)[3][kBin]>(sraw);
    int(*soff)[3] = reinterpret_cast<int(*)[3]>(sraw + kSwBytes);
    T *sq = reinterpret_cast<T *>(sraw + kSwBytes + kOffBytes);
    T(*red)[kRedStride] = reinterpret_cast<T(*)[kRedStride]>(sraw);
    const int ntx = (g.Mt + kBin - 1) / kBin, nty = ntx;
    const int tile = blockIdx.x / kSpreadSplit, part = blockIdx.x % kSpreadSplit;
    const int txi = tile % ntx, tyi = (tile / ntx) % nty, tzi = tile / (ntx * nty);
    const int x0 = txi * kBin, y0 = tyi * kBin, z0 = tzi * kBin;
    const int grp = threadIdx.x >> 4, tl = threadIdx.x & 15;
    const int tz = 2 * (tl >> 2), ty = 2 * (tl & 3);  // this thread's z and y pairs
    const int P = g.P, M3 = g.M3;
    // FP32 window rows fetched as aligned 16-byte chunks (P % 4 == 0); the z rows so only where the
    // support cannot wrap onto itself within a tile (M3 >= P + 8)
    const bool vec_rows = (P & 3) == 0, short_z = M3 < P + kBin;
    T acc[4][kBin];  // [2 dz + dy][x]
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kBin; ++c) acc[r][c] = (T)0;
    f32x2 acc2[4][kBin / 2];  // FP32: the same sums as packed column pairs
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int j = 0; j < kBin / 2; ++j) acc2[r][j] = 0ull;

    // bins whose start indices can reach the tile
    const int bx_lo = max(x0 - P + 1, 0) / kBin, bx_hi = min(x0 + kBin - 1, g.Mt - P) / kBin;
    const int by_lo = max(y0 - P + 1, 0) / kBin, by_hi = min(y0 + kBin - 1, g.Mt - P) / kBin;
    __shared__ int zbl[8], nzb_s;
    __shared__ int rbeg[kSpreadMaxRows], rpre[kSpreadMaxRows + 1];
    __shared__ int sidx[kSpreadBatch];  // record index of each particle of the batch
    if (threadIdx.x == 0) {
        // z bins: the cyclic range of starts [z0 - P + 1, z0 + 7], or all of them on a short z axis;
        // this CTA takes those with (visit count) % kSpreadSplit == part
        const int span = P + kBin - 1;
        const bool allz = span + 2 * kBin > M3;
        int nz = 0, u = 0, zb_iter = 0, zcount = 0;
        while (true) {
            int bz;
            if (allz) {
                if (zb_iter >= g.nbz) break;
                bz = zb_iter++;
            } else {
                if (u >= span) break;
                int s = z0 - P + 1 + u;
                if (s < 0) s += M3;
                if (s >= M3) s -= M3;
                bz = s / kBin;
                u += min((bz + 1) * kBin, M3) - s;
            }
            if ((zcount++ % kSpreadSplit) != part) continue;
            if (nz < 8) zbl[nz++] = bz;
        }
        nzb_s = (bx_lo > bx_hi || by_lo > by_hi) ? 0 : nz;
    }
    __syncthreads();
    const int nyb = by_hi - by_lo + 1;
    const int nrows = min(nzb_s * max(nyb, 0), kSpreadMaxRows);
    if (threadIdx.x < 32) {
        // each (z, y) row of bins is one range of the bin-sorted records; their lengths and offsets in
        // the concatenated list (two rows per lane, one warp scan), loaded in parallel
        int len[2], beg[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = threadIdx.x + 32 * h;
            len[h] = 0;
            beg[h] = 0;
            if (r < nrows) {
                const int row = (zbl[r / nyb] * g.nby + by_lo + r % nyb) * g.nbx;
                beg[h] = bin_start[row + bx_lo];
                len[h] = bin_start[row + bx_hi + 1] - beg[h];
            }
        }
        int inc0 = len[0], inc1 = len[1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int s0 = __shfl_up_sync(0xffffffffu, inc0, o), s1 = __shfl_up_sync(0xffffffffu, inc1, o);
            if ((int)threadIdx.x >= o) {
                inc0 += s0;
                inc1 += s1;
            }
        }
        const int tot0 = __shfl_sync(0xffffffffu, inc0, 31);
        rbeg[threadIdx.x] = beg[0];
        rbeg[threadIdx.x + 32] = beg[1];
        rpre[threadIdx.x] = inc0 - len[0];
        rpre[threadIdx.x + 32] = tot0 + inc1 - len[1];
        if (threadIdx.x == 31) rpre[64] = tot0 + inc1;
    }
    __syncthreads();
    const int total = rpre[nrows];  // rows past nrows have length 0
    const bool any = total > 0;     // the tile saw a particle (the same for every thread of the CTA)
    int rcur = 0;                   // this thread's row (its element of each batch only moves forward)
    static_assert(kSpreadBatch == kSpreadThreads, "one record per thread and batch");
    for (int v0 = 0; v0 < total; v0 += kSpreadBatch) {
        const int nb = min(kSpreadBatch, total - v0);
        __syncthreads();  // previous batch fully consumed
        if ((int)threadIdx.x < nb) {
            const int v = v0 + (int)threadIdx.x, b = threadIdx.x;
            while (rpre[rcur + 1] <= v) ++rcur;
            const int i = rbeg[rcur] + (v - rpre[rcur]);
            sidx[b] = i;
            const PartRec<T> pr = parts[i];
            // support offset of the tile origin per axis; z taken cyclically into [0, M3), so that
            // dz + o needs one wrap (a plain difference misses the wrapped part of the support when
            // M3 < P + 8)
            int dz = z0 - pr.i0[2];
            if (dz < 0) dz += M3;
            soff[b][0] = x0 - pr.i0[0];
            soff[b][1] = y0 - pr.i0[1];
            soff[b][2] = dz;
            sq[b] = pr.q;
        }
        __syncthreads();
        // window values at the tile's 8 offsets: one thread per (particle, axis), i.e. per row
        // e = 3 b + a of sw
        for (int e = threadIdx.x; e < nb * 3; e += kSpreadThreads) {
            const int b = e / 3, a = e - 3 * b;
            const T *wrow = wts + (size_t)sidx[b] * 3 * P + a * P;
            const int base = soff[b][a];
            const T scale = a == 2 ? sq[b] : (T)1;
            if constexpr (sizeof(T) == 4) {
                if (vec_rows && (a < 2 || !short_z)) {
                    // the rows are 16-byte aligned (P % 4 == 0): the 8 offsets lie in three aligned
                    // 4-value chunks from the first offset rounded down, each wholly inside [0, P) or
                    // outside it; on the z axis an offset past M3 - 8 means the wrapped part of the
                    // support, which (M3 >= P + 8) starts before it, at base - M3 in [-7, -1]
                    const int bs = (a == 2 && base > M3 - kBin) ? base - M3 : base;
                    const int c = bs & ~3, sh = bs & 3;
                    float u[12];
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int ck = c + 4 * k;
                        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ck >= 0 && ck < P) t = *reinterpret_cast<const float4 *>(wrow + ck);
                        u[4 * k] = t.x;
                        u[4 * k + 1] = t.y;
                        u[4 * k + 2] = t.z;
                        u[4 * k + 3] = t.w;
                    }
                    float u2[10], w[kBin];
#pragma unroll
                    for (int o = 0; o < 10; ++o) u2[o] = (sh & 2) ? u[o + 2] : u[o];
#pragma unroll
                    for (int o = 0; o < kBin; ++o) w[o] = ((sh & 1) ? u2[o + 1] : u2[o]) * scale;
                    // two 16-byte stores per 32-byte row; rows e and e + 4 (the same banks) store
                    // opposite halves first, so each quarter-warp phase covers the 32 banks once
                    const float4 lo = make_float4(w[0], w[1], w[2], w[3]);
                    const float4 hi = make_float4(w[4], w[5], w[6], w[7]);
                    const int h = (e >> 2) & 1;
                    float4 *dst = reinterpret_cast<float4 *>(&sw[b][a][0]);
                    dst[h] = h ? hi : lo;
                    dst[h ^ 1] = h ? lo : hi;
                    continue;
                }
            }
            T v[kBin];
#pragma unroll
            for (int o = 0; o < kBin; ++o) {
                int rel = base + o;
                if (a == 2 && rel >= M3) rel -= M3;
                v[o] = (rel >= 0 && rel < P) ? wrow[rel] * scale : (T)0;
            }
#pragma unroll
            for (int o = 0; o < kBin; ++o) sw[b][a][o] = v[o];
        }
        __syncthreads();
#pragma unroll 8  // independent particles interleave their shared loads (0.51 -> 0.44 ms at C2)
        for (int b = grp; b < nb; b += kSpreadGroups) {
            const T wz0 = sw[b][2][tz], wz1 = sw[b][2][tz + 1];
            const T wy0 = sw[b][1][ty], wy1 = sw[b][1][ty + 1];
            const T s00 = wz0 * wy0, s01 = wz0 * wy1, s10 = wz1 * wy0, s11 = wz1 * wy1;
            if constexpr (sizeof(T) == 4) {
                // packed pairs of x columns: 16 two-wide FMAs instead of 32
                const float4 xa = *reinterpret_cast<const float4 *>(&sw[b][0][0]);
                const float4 xb = *reinterpret_cast<const float4 *>(&sw[b][0][4]);
                const f32x2 w[4] = {f2_pack(xa.x, xa.y), f2_pack(xa.z, xa.w), f2_pack(xb.x, xb.y),
                                 f2_pack(xb.z, xb.w)};
                const f32x2 sp[4] = {f2_splat(s00), f2_splat(s01), f2_splat(s10), f2_splat(s11)};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int j = 0; j < kBin / 2; ++j) acc2[r][j] = f2_fma(sp[r], w[j], acc2[r][j]);
            } else {
#pragma unroll
                for (int c = 0; c < kBin; ++c) {
                    const T wx = sw[b][0][c];
                    acc[0][c] += s00 * wx;
                    acc[1][c] += s01 * wx;
                    acc[2][c] += s10 * wx;
                    acc[3][c] += s11 * wx;
                }
            }
        }
    }
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int j = 0; j < kBin / 2; ++j) {
                const float2 v = f2_unpack(acc2[r][j]);
                acc[r][2 * j] = v.x;
                acc[r][2 * j + 1] = v.y;
            }
    }
    if (!any) return;  // nothing to add to the zeroed grid
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kBin; ++c) red[grp][(r * kBin + c) * 16 + tl] = acc[r][c];
    __syncthreads();
    // every thread sums 4 of the tile's 512 points over the groups (point p = (z 8 + y) 8 + x, held
    // by thread (z / 2) 4 + y / 2 of each group as its value (z % 2) 2 + y % 2, column x)
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int pidx = (int)threadIdx.x + kSpreadThreads * k;
        const int zz = pidx >> 6, yy = (pidx >> 3) & 7, xx = pidx & 7;
        const int src = (((zz & 1) * 2 + (yy & 1)) * kBin + xx) * 16 + (zz >> 1) * 4 + (yy >> 1);
        T v = (T)0;
#pragma unroll
        for (int q = 0; q < kSpreadGroups; ++q) v += red[q][src];
        const int z = z0 + zz, y = y0 + yy;
        // the grid is zeroed before the launch: points outside every support (exact zeros) add nothing
        if (v != (T)0 && z < M3 && y < g.Mt && x0 + xx < g.Mt) atomicAdd(grid + gidx(z, y, x0 + xx, g.Mt, gnxb(g.Mt)), v);
    }
}

// ------------------------------------------------------------------ gathering (Eqs. 3.11, 3.25)
//
template <typename VT> __device__ __forceinline__ VT make_zero();
template <> __device__ __forceinline__ float4 make_zero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 make_zero<double2>() { return make_double2(0.0, 0.0); }
__device__ __forceinline__ float dotv(const float *w, float4 v) { return w[0] * v.x + w[1] * v.y + w[2] * v.z + w[3] * v.w; }
__device__ __forceinline__ double dotv(const double *w, double2 v) { return w[0] * v.x + w[1] * v.y; }

__device__ __forceinline__ int sm_id()
{
    int v;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(v));
    return v;
}

// Particle handout of the gather, for long particle lists.  The bin-sorted particles form chunks of
// cl consecutive ones, and sequence q is made of the chunks q, q + nseq, q + 2 nseq, ... (one sequence
// per SM, all of them equally long but for the last chunk).  A warp starts on the sequence of its SM, so the warps of one SM read neighbouring supports
// at the same time and find them in L1 (with a fixed stride over the particles, the CTAs of an SM
// worked on unrelated parts of the grid: L1 hit rate 66 %), and all SMs move through the grid together,
// so that the part of the grid in use stays in L2 (one contiguous chunk per SM kept the whole grid in
// use at once: with 10^6 particles on 128 x 128 x 1024 points the L2 hit rate fell to 62 %).  Once
// its sequence is used up a warp moves to the sequence with the most particles left.  Every index is
// handed out once, by an atomic add on the sequence's cursor; no warp waits for another.  A warp's
// current sequence sits in shared memory (st[0]), where it costs the gather's loop no registers.
struct ChunkArgs {
    int *next;   // cursor of each sequence
    int nseq;    // sequences, 0: no handout (warp w takes the particles w, w + warps, ...)
    int nchunk;  // chunks
    int cl;      // chunk length
    FastDiv fcl;
    int n;
};

__device__ __forceinline__ int chunk_claim(const ChunkArgs &c, const int *st, int lane)
{
    return lane == 0 ? atomicAdd(c.next + st[0], 1) : 0;
}

// the particle of the t-th claim on sequence q (n or more once the sequence is used up)
__device__ __forceinline__ int seq_particle(const ChunkArgs &c, int q, int t)
{
    const int j = fdiv(t, c.fcl);
    return (q + c.nseq * j) * c.cl + (t - j * c.cl);
}

__device__ __forceinline__ void chunk_set(int *st, int q, int lane)
{
    __syncwarp();
    if (lane == 0) st[0] = q;
    __syncwarp();
}

// the current sequence is used up: claim from the one with the most left (all cursors read at once,
// in L2, where the atomics act); -1 when every sequence is used up
__device__ __forceinline__ int chunk_refill(const ChunkArgs &c, int *st, int lane)
{
    while (true) {
        int left = 0, best = -1;
        for (int q = lane; q < c.nseq; q += 32) {
            // particles of sequence q: its chunks, the last chunk of the list possibly short
            const int cnt = q < c.nchunk ? (c.nchunk - 1 - q) / c.nseq + 1 : 0;
            int len = cnt * c.cl;
            if (cnt > 0 && (c.nchunk - 1) % c.nseq == q) len -= c.nchunk * c.cl - c.n;
            const int l = len - __ldcg(c.next + q);
            if (l > left) {
                left = l;
                best = q;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const int ol = __shfl_xor_sync(0xffffffffu, left, o), ob = __shfl_xor_sync(0xffffffffu, best, o);
            if (ol > left || (ol == left && ob > best)) {
                left = ol;
                best = ob;
            }
        }
        if (left <= 0) return -1;
        chunk_set(st, best, lane);
        const int pi = seq_particle(c, best, __shfl_sync(0xffffffffu, chunk_claim(c, st, lane), 0));
        if (pi < c.n) return pi;
    }
}

// the particle of a claim made earlier, else one of another sequence, else -1
__device__ __forceinline__ int chunk_take(const ChunkArgs &c, int *st, int ticket, int lane)
{
    const int pi = seq_particle(c, st[0], __shfl_sync(0xffffffffu, ticket, 0));
    return pi < c.n ? pi : chunk_refill(c, st, lane);
}

// Vectorised gathering on the x-blocked grid, for supports of P <= PC points (the loop shapes follow
// PC, the rows and z levels past P are skipped).  A particle's x support [i0, i0 + P) lies in NB blocks
// of kXB points starting at block i0 / kXB; a warp request covers two blocks x RG rows x the block's
// VPB 16-byte vectors (32 lanes: lane = (block of the pair, row, vector)), i.e. two 256-byte runs of
// consecutive rows, whole 128-byte lines.  Each lane holds the x window values of its V points (zero
// outside the support) for each pair of blocks and accumulates, per row, sum wx H and sum wx dx H,
// weighted by the row's y values (wy, wy dy); the z rows are weighted at the end of each z level.
// FP32 is compiled for four CTAs per SM (64 registers): with the loads of four z levels in flight the
// kernel is latency-bound, and 32 resident warps beat 24 (C2 alone 0.356 against 0.407 ms).
template <typename T, int PC, bool EXACT, bool HANDOUT>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? (PC > 24 ? 3 : 4) : 1) k_gather_vec(Geo g, int n, const PartRec<T> *__restrict__ parts,
                                                    const T *__restrict__ wts, const T *__restrict__ grid,
                                                    double *__restrict__ phi, double *__restrict__ frc,
                                                    int flags, GatherScale sc, ChunkArgs ca)
{
    constexpr int V = 16 / sizeof(T);                    // values per 16-byte vector
    constexpr int VPB = kXB / V;                         // vectors per block row
    constexpr int RG = 32 / (2 * VPB);                   // rows per request
    constexpr int NB = (PC + kXB - 1 + kXB - 1) / kXB;   // blocks a support can touch
    constexpr int NBP = (NB + 1) / 2;                    // block pairs
    constexpr int NRG = (PC + RG - 1) / RG;              // row groups
    constexpr int NJ = NRG * RG;                         // y rows padded to a multiple of RG
    using VecT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    __shared__ T sy[8][2][NJ];
    __shared__ T sz[8][2][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int bi = lane / (RG * VPB), rem = lane - bi * (RG * VPB);
    const int r = rem / VPB, qv = rem - r * VPB;  // row within the request, vector within the block row
    const int nxb = gnxb(g.Mt);
    const int P = EXACT ? PC : g.P;  // support width, P <= PC (a compile-time trip count where P = PC)
    __shared__ int sst[8];
    int *st = sst + wib;
    const int warps_total = gridDim.x * (blockDim.x >> 5);
    int pi = blockIdx.x * (blockDim.x >> 5) + wib;
    if (HANDOUT) {
        chunk_set(st, sm_id() % ca.nseq, lane);
        pi = chunk_take(ca, st, chunk_claim(ca, st, lane), lane);
    }
    while (pi >= 0 && pi < n) {
        // the next particle, claimed now and read after this one
        const int ticket = HANDOUT ? chunk_claim(ca, st, lane) : 0;
        const PartRec<T> pr = parts[pi];
        const T *w = wts + (size_t)pi * 3 * P;
        for (int j = lane; j < NJ; j += 32) {
            T wy = 0, wyd = 0;
            if (j < P) {
                wy = w[P + j];
                wyd = wy * (pr.g[1] - (T)(j - g.c));
            }
            sy[wib][0][j] = wy;
            sy[wib][1][j] = wyd;
        }
        if (lane < P) {
            const T wz = w[2 * P + lane];
            sz[wib][0][lane] = wz;
            sz[wib][1][lane] = wz * (pr.g[2] - (T)(lane - g.c));
        }
        // this lane's V x points in each block pair: x = (xb0 + 2 bp + bi) kXB + V qv + e
        const int xb0 = pr.i0[0] / kXB;
        T wx[NBP][V], wxd[NBP][V];
        bool ld[NBP];
        int loff[NBP];  // offset of this lane's first vector inside a z plane, row i0y + r
#pragma unroll
        for (int bp = 0; bp < NBP; ++bp) {
            const int blk = xb0 + 2 * bp + bi;
            // a block is read when it exists and holds at least one support point
            ld[bp] = blk < nxb && blk * kXB < pr.i0[0] + P;
            loff[bp] = (blk * g.Mt + pr.i0[1] + r) * kXB + V * qv;
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int rel = blk * kXB + V * qv + e - pr.i0[0];
                const bool in = rel >= 0 && rel < P;
                wx[bp][e] = in ? w[rel] : (T)0;
                wxd[bp][e] = in ? wx[bp][e] * (pr.g[0] - (T)(rel - g.c)) : (T)0;
            }
        }
        __syncwarp();
        T aphi = 0, afx = 0, afy = 0, afz = 0;
        const size_t plane = (size_t)nxb * g.Mt * kXB;
#pragma unroll 4  // several z levels' loads in flight
        for (int k = 0; k < P; ++k) {
            int zk = pr.i0[2] + k;
            if (zk >= g.M3) zk -= g.M3;
            const T *gk = grid + (size_t)zk * plane;
            T a = 0, b = 0, c = 0;
#pragma unroll
            for (int rg = 0; rg < NRG; ++rg) {
                const int j = rg * RG + r;
                const T wy = sy[wib][0][j], wyd = sy[wib][1][j];
#pragma unroll
                for (int bp = 0; bp < NBP; ++bp) {
                    VecT v = make_zero<VecT>();
                    if (ld[bp] && j < P) v = *reinterpret_cast<const VecT *>(gk + loff[bp] + rg * RG * kXB);
                    const T s1 = dotv(wx[bp], v), s2 = dotv(wxd[bp], v);
                    a += wy * s1;
                    b += wy * s2;
                    c += wyd * s1;
                }
            }
            const T wz = sz[wib][0][k], wzd = sz[wib][1][k];
            aphi += wz * a;
            afx += wz * b;
            afy += wz * c;
            afz += wzd * a;
        }
        const T vphi = warp_sum(aphi), vfx = warp_sum(afx), vfy = warp_sum(afy), vfz = warp_sum(afz);
        if (lane == 0) {
            const double qd = (double)pr.q;
            double ph = sc.phi * (double)vphi;
            if (flags & 1) ph += -2.0 * g.xi / sqrt(kPi) * qd;
            phi[pr.orig] = ph;
            const double qf = (flags & 2) ? 1.0 : qd;
            frc[3 * pr.orig + 0] = qf * sc.fxy * (double)vfx;
            frc[3 * pr.orig + 1] = qf * sc.fxy * (double)vfy;
            frc[3 * pr.orig + 2] = qf * sc.fz * (double)vfz;
        }
        __syncwarp();
        pi = HANDOUT ? chunk_take(ca, st, ticket, lane) : pi + warps_total;
    }
}

// ------------------------------------------------------------------ outputs and energy
// phi, F in caller order (the grid path's, plus the real space's when it ran on its own stream)
// and the per-block partial energies.
__global__ void k_finalize(int n, const double *__restrict__ xyzq, const double *__restrict__ phi_int,
                           const double *__restrict__ frc_int, const double *__restrict__ phi_add,
                           const double *__restrict__ frc_add, double *__restrict__ phi,
                           double *__restrict__ frc, double *__restrict__ epart)
{
    double e = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double ph = phi_int[i];
        if (phi_add) ph += phi_add[i];
        e += xyzq[4 * i + 3] * ph;
        if (phi) phi[i] = ph;
        if (frc) {
            double f0 = frc_int[3 * i], f1 = frc_int[3 * i + 1], f2 = frc_int[3 * i + 2];
            if (frc_add) {
                f0 += frc_add[3 * i];
                f1 += frc_add[3 * i + 1];
                f2 += frc_add[3 * i + 2];
            }
            frc[3 * i] = f0;
            frc[3 * i + 1] = f1;
            frc[3 * i + 2] = f2;
        }
    }
    __shared__ double ws[32];
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) epart[blockIdx.x] = v;
    }
}

__global__ void k_energy_final(const double *__restrict__ epart, int nparts, double *__restrict__ energy)
{
    __shared__ double ws[32];
    double e = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) e += epart[i];
    e = warp_sum(e);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) *energy = 0.5 * v;
    }
}

// Adjoint of phi (see se1p_eval_vjp): grad_q = phi[v], grad_x = -(v E[q] + q E[v]).
__global__ void k_vjp_combine(int n, const double *__restrict__ q, const double *__restrict__ v,
                              const double *__restrict__ Eq, const double *__restrict__ phiv,
                              const double *__restrict__ Ev, double *__restrict__ grad_x,
                              double *__restrict__ grad_q)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (grad_q) grad_q[i] = phiv[i];
    if (grad_x) {
        const double vi = v[i], qi = q[i];
#pragma unroll
        for (int d = 0; d < 3; ++d) grad_x[3 * i + d] = -(vi * Eq[3 * i + d] + qi * Ev[3 * i + d]);
    }
}

// Conversions between a plan's grid (T, x-blocks) and the [z][y][x] FP64 grids of the single-step
// entry points; i runs over the M3 x Mt x Mt points in [z][y][x] order.
template <typename T>
__global__ void k_grid_to_user(int M3, int Mt, const T *__restrict__ src, double *__restrict__ dst, double scale)
{
    const size_t n = (size_t)M3 * Mt * Mt;
    const int nxb = gnxb(Mt);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mt), y = (int)((i / Mt) % Mt), z = (int)(i / ((size_t)Mt * Mt));
        dst[i] = (double)src[gidx(z, y, x, Mt, nxb)] * scale;
    }
}

template <typename T>
__global__ void k_grid_from_user(int M3, int Mt, const double *__restrict__ src, T *__restrict__ dst)
{
    const size_t n = (size_t)M3 * Mt * Mt;
    const int nxb = gnxb(Mt);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mt), y = (int)((i / Mt) % Mt), z = (int)(i / ((size_t)Mt * Mt));
        dst[gidx(z, y, x, Mt, nxb)] = (T)src[i];
    }
}

// Triply periodic plans grid on the extended grid (Mt = M + P, origin -P h/2) and transform the
// M-periodic grid.  Extended point i sits at (i - P/2) h, periodic point j at j h, so i maps to
// j = (i - P/2) mod M.  Fold: each periodic point sums its (at most four) extended preimages in a
// fixed order; unfold: each extended point copies its periodic image.
template <typename T>
__global__ void k_fold(int M3, int Mt, int Mf, int sh, const T *__restrict__ ext, T *__restrict__ per)
{
    const size_t total = (size_t)M3 * Mf * Mf;
    const int nxbt = gnxb(Mt), nxbf = gnxb(Mf);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int jx = (int)(i % Mf), jy = (int)((i / Mf) % Mf), z = (int)(i / ((size_t)Mf * Mf));
        T acc = (T)0;
        for (int iy = (jy + sh) % Mf; iy < Mt; iy += Mf)
            for (int ix = (jx + sh) % Mf; ix < Mt; ix += Mf) acc += ext[gidx(z, iy, ix, Mt, nxbt)];
        per[gidx(z, jy, jx, Mf, nxbf)] = acc;
    }
}

template <typename T>
__global__ void k_unfold(int M3, int Mt, int Mf, int sh, const T *__restrict__ per, T *__restrict__ ext)
{
    const size_t total = (size_t)M3 * Mt * Mt;
    const int nxbt = gnxb(Mt), nxbf = gnxb(Mf);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % Mt), iy = (int)((i / Mt) % Mt), z = (int)(i / ((size_t)Mt * Mt));
        const int jx = (ix - sh + Mf) % Mf, jy = (iy - sh + Mf) % Mf;  // sh = P/2 <= Mf
        ext[gidx(z, iy, ix, Mt, nxbt)] = per[gidx(z, jy, jx, Mf, nxbf)];
    }
}

// CTAs for n items of bs threads; kernels with one thread per item and no grid-stride loop
// pass an uncapped limit
inline int blocks_for(size_t n, int bs, int cap = 1 << 20)
{
    size_t b = (n + bs - 1) / bs;
    if (b < 1) b = 1;
    return (int)(b > (size_t)cap ? cap : b);
}

}  // namespace

// ------------------------------------------------------------------ launchers
template <typename T>
void launch_pack(se1p_plan *p, int n, const double *x, const double *q, cudaStream_t s, int check_neutral)
{
    const Geo &g = p->geo;
    cudaMemsetAsync(p->b.counts, 0, sizeof(int) * (g.nbins + g.ncells), s);
    cudaMemsetAsync(p->b.sums, 0, sizeof(double) * 2, s);
    if (n > 0)
        k_pack<T><<<blocks_for(n, 256, 0x7fffffff), 256, 0, s>>>(g, n, x, q, p->b.xyzq, p->b.bin_key, p->b.cell_key,
                                                       p->b.counts, p->b.counts + g.nbins, p->b.sums,
                                                       p->b.status);
    if (g.ncells <= 16 * kScanChunk) {
        k_scan<<<2, 1024, 0, s>>>(g.nbins, g.ncells, p->b.counts, p->b.starts, p->b.cursors, p->b.sums,
                                  p->b.status, check_neutral);
    } else {
        // many cells: one block scans the bins, three launches scan the cells
        k_scan<<<1, 1024, 0, s>>>(g.nbins, g.ncells, p->b.counts, p->b.starts, p->b.cursors, p->b.sums,
                                  p->b.status, check_neutral);
        const int nblk = (g.ncells + kScanChunk - 1) / kScanChunk;  // <= kScanTmp (2^22 cells at most)
        const int *cc = p->b.counts + g.nbins;
        k_scan_sums<<<nblk, kScanThreads, 0, s>>>(g.ncells, cc, p->b.scan_tmp);
        k_scan_offsets<<<1, kScanThreads, 0, s>>>(nblk, p->b.scan_tmp);
        k_scan_write<<<nblk, kScanThreads, 0, s>>>(g.ncells, cc, p->b.scan_tmp, p->b.starts + g.nbins + 1,
                                                   p->b.cursors + g.nbins);
    }
}

template <typename T> void launch_sort_scatter(se1p_plan *p, int n, cudaStream_t s)
{
    const Geo &g = p->geo;
    if (n <= 0) return;
    // one thread per particle (no grid-stride loop, so no cap on the CTA count); per-warp buffers of
    // 32 rows of 3P + 1 values: at most 24.8 KB per CTA (P <= 32)
    const int nt = sizeof(T) == sizeof(float) ? kScatterThreads : kScatterThreads / 2;
    const size_t sm = sizeof(T) * (size_t)nt * (3 * g.P + 1);
    k_scatter<T><<<blocks_for(n, nt, 0x7fffffff), nt, sm, s>>>(g, n, p->b.xyzq, p->b.bin_key, p->b.cell_key,
                                                      p->b.cursors, p->b.cursors + g.nbins,
                                                      (PartRec<T> *)p->b.parts, (T *)p->b.wts,
                                                      (CellRec<T> *)p->b.cells);
}

template <typename T> void launch_spread(se1p_plan *p, cudaStream_t s)
{
    const Geo &g = p->geo;
    const int nt = (g.Mt + kBin - 1) / kBin;
    const int ntz = (g.M3 + kBin - 1) / kBin;
    cudaMemsetAsync(p->b.grid, 0, sizeof(T) * grid_points(g.M3, g.Mt), s);
    k_spread<T><<<nt * nt * ntz * kSpreadSplit, kSpreadThreads, 0, s>>>(g, p->b.starts, (const PartRec<T> *)p->b.parts,
                                              (const T *)p->b.wts, (T *)p->b.grid);
}

template <typename T>
using GatherKernel = void (*)(Geo, int, const PartRec<T> *, const T *, const T *, double *, double *, int, GatherScale,
                              ChunkArgs);

// the x-blocked grid keeps every block row 16-byte aligned: vector loads for every P (the smallest
// compiled bound that holds it; 64 systems with P = 18 gathered 4x faster per point than with
// scalar loads)
template <typename T, bool H> GatherKernel<T> gather_kernel_h(int P)
{
    if (P == 24) return k_gather_vec<T, 24, true, H>;
    if (P == 16) return k_gather_vec<T, 16, true, H>;
    if (P == 12) return k_gather_vec<T, 12, true, H>;
    if (P < 12) return k_gather_vec<T, 12, false, H>;
    if (P < 16) return k_gather_vec<T, 16, false, H>;
    if (P < 24) return k_gather_vec<T, 24, false, H>;
    return k_gather_vec<T, 32, false, H>;
}
template <typename T> GatherKernel<T> gather_kernel(int P, bool handout)
{
    return handout ? gather_kernel_h<T, true>(P) : gather_kernel_h<T, false>(P);
}

constexpr int kGatherWarps = 8;  // warps per CTA, one particle each at a time
// the handout pays where each resident warp gathers at least this many particles; shorter lists take
// one particle per warp, with no atomics (64 systems of 1000 to 50 000 particles: 15.10 against
// 14.63 ms with every list handed out)
constexpr int kGatherHandoutPerWarp = 16;
// longest chunk: the SMs' chunks together make the part of the grid in use at once (N = 10^6 on
// 160^2 x 1024 points, gather alone: power-of-two chunks of 64 / 1024 / 4096 took 3.35 / 3.22 / 3.37 ms;
// one contiguous chunk per SM 3.52 ms, the whole grid in use and the L2 hit rate down to 62 %)
constexpr int kGatherChunkMax = 1024;

template <typename T>
void launch_gather(se1p_plan *p, int n, const void *grid, double *phi, double *frc, int flags, cudaStream_t s)
{
    if (n <= 0) return;
    ChunkArgs ca;
    ca.next = p->b.gchunk;
    ca.n = n;
    ca.nseq = 0;
    ca.nchunk = 0;
    ca.cl = 1;
    int blocks = (n + kGatherWarps - 1) / kGatherWarps;  // one particle per warp
    if ((long long)n >= (long long)kGatherHandoutPerWarp * kGatherWarps * p->gather_ctas) {
        // as many CTAs as are resident at once; every sequence the same number of chunks of at most
        // kGatherChunkMax particles (N = 10^5 on 96^2 x 64 points: one chunk of 658 per SM; N = 10^6 on
        // 160^2 x 1024: seven of 940)
        blocks = p->gather_ctas;
        const int nsq = std::min(p->nsm, kGatherChunks);
        const int rounds = (n + nsq * kGatherChunkMax - 1) / (nsq * kGatherChunkMax);
        ca.cl = (n + nsq * rounds - 1) / (nsq * rounds);
        ca.nchunk = (n + ca.cl - 1) / ca.cl;
        ca.nseq = std::min(nsq, ca.nchunk);
    }
    ca.fcl = make_fastdiv((unsigned)ca.cl);
    const Geo &g = p->geo;
    // FP64 constants applied to the FP32 sums: quadrature weight h^3, the window
    // normalisation of the gather (and of the spread when the grid is this plan's own
    // unnormalised spread, flag bit 2), and for the force 4 xi^2 / eta times the grid
    // step that turns the offsets (grid units) into lengths
    const double w3 = g.wnorm_xy * g.wnorm_xy * g.wnorm_z;
    GatherScale sc;
    sc.phi = g.h * g.h * g.hz * w3 * ((flags & 4) ? w3 : 1.0);
    sc.fxy = sc.phi * 4.0 * g.xi * g.xi / g.eta * g.h;
    sc.fz = sc.phi * 4.0 * g.xi * g.xi / g.etaz * g.hz;
    if (ca.nseq > 0) cudaMemsetAsync(p->b.gchunk, 0, sizeof(int) * (size_t)ca.nseq, s);
    gather_kernel<T>(g.P, ca.nseq > 0)<<<blocks, 32 * kGatherWarps, 0, s>>>(g, n, (const PartRec<T> *)p->b.parts,
                                                               (const T *)p->b.wts, (const T *)grid, phi, frc, flags,
                                                               sc, ca);
}

void launch_vjp_combine(int n, const double *q, const double *v, const double *Eq, const double *phiv,
                        const double *Ev, double *grad_x, double *grad_q, cudaStream_t s)
{
    if (n > 0) k_vjp_combine<<<blocks_for(n, 256, 0x7fffffff), 256, 0, s>>>(n, q, v, Eq, phiv, Ev, grad_x, grad_q);
}

void launch_finalize(se1p_plan *p, int n, double *phi, double *frc, double *energy, cudaStream_t s,
                     const double *phi_add, const double *frc_add)
{
    k_finalize<<<kEnergyBlocks, 256, 0, s>>>(n, p->b.xyzq, p->b.phi_int, p->b.frc_int, phi_add, frc_add, phi, frc,
                                             p->b.epart);
    if (energy) k_energy_final<<<1, 256, 0, s>>>(p->b.epart, kEnergyBlocks, energy);
}

template <typename T>
void launch_grid_to_double(se1p_plan *p, const void *src, double *dst, double scale, cudaStream_t s)
{
    const size_t n = (size_t)p->M3 * p->Mt * p->Mt;
    k_grid_to_user<T><<<blocks_for(n, 256, 4096), 256, 0, s>>>(p->M3, p->Mt, (const T *)src, dst, scale);
}

template <typename T> void launch_grid_from_double(se1p_plan *p, const double *src, void *dst, cudaStream_t s)
{
    const size_t n = (size_t)p->M3 * p->Mt * p->Mt;
    k_grid_from_user<T><<<blocks_for(n, 256, 4096), 256, 0, s>>>(p->M3, p->Mt, src, (T *)dst);
}

// the number of CTAs of this plan's handout gather resident at once (a preference for a small
// shared-memory carveout left room for one CTA per SM: 8 KB, 8 warps)
template <typename T> int configure_particle_kernels(se1p_plan *p)
{
    const GatherKernel<T> k = gather_kernel<T>(p->geo.P, true);
    int nsm = 0, occ = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 32 * kGatherWarps, 0) != cudaSuccess) return 1;
    p->nsm = std::max(nsm, 1);
    p->gather_ctas = p->nsm * std::max(occ, 1);
    return 0;
}

template <typename T> void launch_fold(se1p_plan *p, cudaStream_t s)
{
    const size_t n = (size_t)p->M3 * p->Mf * p->Mf;
    k_fold<T><<<blocks_for(n, 256, 152 * 16), 256, 0, s>>>(p->M3, p->Mt, p->Mf, p->geo.P / 2, (const T *)p->b.grid,
                                                           (T *)p->b.gridf);
}

template <typename T> void launch_unfold(se1p_plan *p, cudaStream_t s)
{
    const size_t n = (size_t)p->M3 * p->Mt * p->Mt;
    k_unfold<T><<<blocks_for(n, 256, 152 * 16), 256, 0, s>>>(p->M3, p->Mt, p->Mf, p->geo.P / 2,
                                                             (const T *)p->b.gridf, (T *)p->b.grid);
}

#define SE1P_INST(T)                                                                                        \
    template void launch_pack<T>(se1p_plan *, int, const double *, const double *, cudaStream_t, int);     \
    template void launch_sort_scatter<T>(se1p_plan *, int, cudaStream_t);                                   \
    template void launch_spread<T>(se1p_plan *, cudaStream_t);                                              \
    template void launch_gather<T>(se1p_plan *, int, const void *, double *, double *, int, cudaStream_t);  \
    template void launch_grid_to_double<T>(se1p_plan *, const void *, double *, double, cudaStream_t);           \
    template void launch_grid_from_double<T>(se1p_plan *, const double *, void *, cudaStream_t);           \
    template int configure_particle_kernels<T>(se1p_plan *);                                               \
    template void launch_fold<T>(se1p_plan *, cudaStream_t);                                                \
    template void launch_unfold<T>(se1p_plan *, cudaStream_t);
SE1P_INST(float)
SE1P_INST(double)
#undef SE1P_INST

}  // namespace se1p
