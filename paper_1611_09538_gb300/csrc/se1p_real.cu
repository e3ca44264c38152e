// Real-space part of the Ewald1P sum (Eq. 2.2) and its force (Eq. 3.22) over
// a cell list (Section 3: linked cells no smaller than rc, z images by
// unwrapped neighbour-cell indices).
#include <cuda_runtime.h>
#include <math.h>

#include "se1p_plan.h"

namespace se1p {

namespace {

template <typename T> __device__ __forceinline__ T erfc_t(T v);
template <> __device__ __forceinline__ float erfc_t<float>(float v) { return erfcf(v); }
template <> __device__ __forceinline__ double erfc_t<double>(double v) { return erfc(v); }
template <typename T> __device__ __forceinline__ T exp_t(T v);
template <> __device__ __forceinline__ float exp_t<float>(float v) { return expf(v); }
template <> __device__ __forceinline__ double exp_t<double>(double v) { return exp(v); }

constexpr int kRealThreads = 128;

// One CTA per target cell.  Targets are taken kRealThreads at a time; sources
// of each of the 27 neighbour cells are staged through shared memory.  Pair
// distances use cell-relative coordinates plus the (exact) cell offset, and
// per-chunk partial sums in T are added into FP64 accumulators.
template <typename T>
__global__ void __launch_bounds__(kRealThreads) k_real(Geo g, const int *__restrict__ cell_start,
                                                        const CellRec<T> *__restrict__ cells,
                                                        double *__restrict__ phi, double *__restrict__ frc,
                                                        int accumulate)
{
    __shared__ CellRec<T> src[kRealThreads];
    const int c = blockIdx.x;
    const int cx = c % g.ncx, cy = (c / g.ncx) % g.ncy, cz = c / (g.ncx * g.ncy);
    const int tbeg = cell_start[c], tend = cell_start[c + 1];
    const T xi = (T)g.xi, rc2 = (T)g.rc2;
    const T two_xi_sqpi = (T)(2.0 * g.xi / sqrt(kPi));
    const T xi2 = (T)(g.xi * g.xi);
    for (int t0 = tbeg; t0 < tend; t0 += kRealThreads) {
        const int t = t0 + threadIdx.x;
        const bool valid = t < tend;
        CellRec<T> me;
        if (valid) me = cells[t];
        else {
            me.lx = me.ly = me.lz = me.q = me.ex = me.ey = me.ez = (T)0;
            me.orig = -1;
        }
        double aphi = 0, afx = 0, afy = 0, afz = 0;
        for (int nb = 0; nb < 27; ++nb) {
            const int dcx = nb % 3 - 1, dcy = (nb / 3) % 3 - 1, dcz = nb / 9 - 1;
            const int nx = cx + dcx, ny = cy + dcy, nzu = cz + dcz;
            if (nx < 0 || nx >= g.ncx || ny < 0 || ny >= g.ncy) continue;
            int nz = nzu % g.ncz;
            if (nz < 0) nz += g.ncz;
            const int sc = (nz * g.ncy + ny) * g.ncx + nx;
            // cell offset -dc * cs as hi + lo in T
            const double oxd = -dcx * g.cs[0], oyd = -dcy * g.cs[1], ozd = -dcz * g.cs[2];
            const T ox = (T)oxd, oy = (T)oyd, oz = (T)ozd;
            const T oxl = (T)(oxd - (double)ox), oyl = (T)(oyd - (double)oy), ozl = (T)(ozd - (double)oz);
            const int sbeg = cell_start[sc], send = cell_start[sc + 1];
            for (int s0 = sbeg; s0 < send; s0 += kRealThreads) {
                const int ns = min(kRealThreads, send - s0);
                __syncthreads();
                if (threadIdx.x < ns) src[threadIdx.x] = cells[s0 + threadIdx.x];
                __syncthreads();
                if (!valid) continue;
                T pphi = 0, pfx = 0, pfy = 0, pfz = 0;
                for (int j = 0; j < ns; ++j) {
                    const CellRec<T> sr = src[j];
                    T dx = (me.lx - sr.lx) + ox, dy = (me.ly - sr.ly) + oy, dz = (me.lz - sr.lz) + oz;
                    if constexpr (sizeof(T) < sizeof(double)) {
                        dx += (me.ex - sr.ex) + oxl;
                        dy += (me.ey - sr.ey) + oyl;
                        dz += (me.ez - sr.ez) + ozl;
                    }
                    const T r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 > rc2) continue;
                    if (dcz == 0 && s0 + j == t) continue;  // the target itself (alpha = 0)
                    const T r = sqrt(r2);
                    const T e = erfc_t<T>(xi * r) / r;
                    pphi += sr.q * e;
                    const T fs = sr.q * (two_xi_sqpi * exp_t<T>(-xi2 * r2) + e) / r2;
                    pfx += fs * dx;
                    pfy += fs * dy;
                    pfz += fs * dz;
                }
                aphi += (double)pphi;
                afx += (double)pfx;
                afy += (double)pfy;
                afz += (double)pfz;
            }
        }
        if (valid) {
            const double qm = (double)me.q;
            const int o = me.orig;
            if (accumulate) {
                phi[o] += aphi;
                frc[3 * o] += qm * afx;
                frc[3 * o + 1] += qm * afy;
                frc[3 * o + 2] += qm * afz;
            } else {
                phi[o] = aphi;
                frc[3 * o] = qm * afx;
                frc[3 * o + 1] = qm * afy;
                frc[3 * o + 2] = qm * afz;
            }
        }
    }
}

}  // namespace

template <typename T> void launch_real_space(se1p_plan *p, double *phi, double *frc, int accumulate, cudaStream_t s)
{
    const Geo &g = p->geo;
    k_real<T><<<g.ncells, kRealThreads, 0, s>>>(g, p->b.starts + g.nbins + 1, (const CellRec<T> *)p->b.cells, phi,
                                                frc, accumulate);
}

template void launch_real_space<float>(se1p_plan *, double *, double *, int, cudaStream_t);
template void launch_real_space<double>(se1p_plan *, double *, double *, int, cudaStream_t);

}  // namespace se1p
