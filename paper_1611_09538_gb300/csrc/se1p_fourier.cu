// Fourier-side kernels of the SE1P path: the adaptive FFT (Algorithm 2), the
// scaling step (Eq. 3.5 with the Green's functions of Eqs. 3.6-3.10) and the
// inverse adaptive FFT (Algorithm 3).
//
// Passes (all transforms are hand-written Stockham FFTs in shared memory):
//   z  : real grid -> k3 = 1..K3-1 complex slabs (and the k3 = 0 slab summed in FP64)
//   xf : per slab row, zero-pad Mt -> ns and FFT along x            (ns = n0, nI or Mt)
//   y  : per slab column, zero-pad Mt -> ns, FFT along y, multiply by the
//        symbol, inverse FFT, keep the Mt spreading rows            (Algorithm 3 step 2-3 crop)
//   xi : per slab row, inverse FFT along x, keep Mt points
//   zi : Hermitian completion along z and inverse FFT -> real grid
// The k3 = 0 slab (Vico-truncated 2-D kernel) always runs in FP64.
#include <cuda_runtime.h>
#include <math.h>

#include "se1p_plan.h"

namespace se1p {

namespace {

__device__ __forceinline__ int signed_index(int i, int n) { return i <= (n - 1) / 2 ? i : i - n; }

// ---- z forward on pencil pairs: the real pencils 2j and 2j + 1 of a row form one complex
// pencil H[2j] + i H[2j + 1] (one aligned two-element load); their spectra follow from its FFT Z by
// Hermitian symmetry, X_2j[k] = (Z[k] + conj Z[-k]) / 2 and X_2j+1[k] = (Z[k] - conj Z[-k]) / 2i.
// CTA = (y, chunk of xp pairs); half the FFT work and shared memory per real pencil.
template <typename T> struct Pair2;
template <> struct Pair2<float> { using type = float2; };
template <> struct Pair2<double> { using type = double2; };

// With a tensor map (tma != 0) the CTA's M3 x 2 xp real values arrive by bulk tensor copies (boxes of
// the x-blocked grid, blocks beyond the row filled with zeros, padding points holding zeros) that land
// in shared memory exactly as the complex pencils: value (z, x = 2 (j0 + pp) + r) at a[z xp + pp], part r.
// The wait on them is bounded (spin_limit polls); a CTA that gives up records FLAG_TIMEOUT in *status,
// waits for its copies to land (bounded as well) and returns without writing results.
template <typename T>
__global__ void k_zfwd_pair(int M3, int Mt, int K3, FftDesc d, const Tw<T> *__restrict__ tw, int xp, FastDiv fxp,
                            const T *__restrict__ grid, Cx<T> *__restrict__ zspec, double *__restrict__ slab0,
                            const __grid_constant__ CUtensorMap tm, int tma, int zbox, int *__restrict__ status,
                            long long spin_limit)
{
    using V2 = typename Pair2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *b = a + (size_t)M3 * xp;
    // pencils 2j and 2j + 1; for odd Mt the last pair's second pencil is x = Mt, the x-blocked grid's
    // zero padding, whose spectra are not stored
    const int npair = (Mt + 1) / 2, nxc = (npair + xp - 1) / xp;
    const int y = blockIdx.x / nxc, j0 = (blockIdx.x % nxc) * xp;
    if (tma) {
        const unsigned bar_a = smem_addr(&bar);
        if (threadIdx.x == 0) {
            mbar_init(bar_a, 1);
            mbar_expect_tx(bar_a, (unsigned)((size_t)M3 * xp * sizeof(Cx<T>)));
            const int x0 = 2 * j0;  // first real pencil: block x0 / 8, offset x0 % 8 inside it
            for (int z0 = 0; z0 < M3; z0 += zbox)
                tma_load_4d(smem_addr(a + (size_t)z0 * xp), &tm, x0 & (kXB - 1), y, x0 / kXB, z0, bar_a);
        }
        __syncthreads();  // the barrier is initialised before anyone polls it
        const bool late = !mbar_wait(bar_a, 0, spin_limit);
        if (__syncthreads_or(late)) {
            if (threadIdx.x == 0) atomicOr(status, FLAG_TIMEOUT);
            mbar_wait(bar_a, 0, kDrainPolls);
            __syncthreads();
            return;
        }
    } else {
        for (int e = threadIdx.x; e < M3 * xp; e += blockDim.x) {
            const int z = fdiv(e, fxp), pp = e - z * xp, j = j0 + pp;
            Cx<T> v = cx<T>((T)0, (T)0);
            if (j < npair) {
                const V2 h = *reinterpret_cast<const V2 *>(grid + gidx(z, y, 2 * j, Mt, gnxb(Mt)));  // a pair never straddles a block
                v = cx<T>(h.x, h.y);
            }
            a[e] = v;
        }
        __syncthreads();
    }
    // k3 = 0: each pencil's z sum to FP64 accuracy, as in k_zfwd (real part: pencil 2j, imaginary: 2j + 1)
    {
        __shared__ double part[2][256];
        const int G = blockDim.x / xp;  // xp is a power of 2 <= 32 that divides blockDim (256)
        const int g = threadIdx.x / xp, pp = threadIdx.x - g * xp;
        double sre = 0.0, sim = 0.0;
        if constexpr (sizeof(T) == sizeof(double)) {
            for (int z = g; z < M3; z += G) {
                sre += (double)a[z * xp + pp].re;
                sim += (double)a[z * xp + pp].im;
            }
        } else {
            float hr = 0.0f, lr = 0.0f, hi = 0.0f, li = 0.0f;
            for (int z = g; z < M3; z += G) {
                const Cx<float> v = a[z * xp + pp];
                const float tr = hr + v.re, br = tr - hr;
                lr += (hr - (tr - br)) + (v.re - br);
                hr = tr;
                const float ti = hi + v.im, bi = ti - hi;
                li += (hi - (ti - bi)) + (v.im - bi);
                hi = ti;
            }
            sre = (double)hr + (double)lr;
            sim = (double)hi + (double)li;
        }
        part[0][threadIdx.x] = sre;
        part[1][threadIdx.x] = sim;
        __syncthreads();
        if (g == 0 && j0 + pp < npair) {
            double tr = 0.0, ti = 0.0;
            for (int k = 0; k < G; ++k) {
                tr += part[0][k * xp + pp];
                ti += part[1][k * xp + pp];
            }
            slab0[(size_t)y * Mt + 2 * (j0 + pp)] = tr;
            if (2 * (j0 + pp) + 1 < Mt) slab0[(size_t)y * Mt + 2 * (j0 + pp) + 1] = ti;
        }
    }
    __syncthreads();
    Cx<T> *res = fft_smem<T>(a, b, d, xp, fxp, 1, xp, tw, -1);
    for (int e = threadIdx.x; e < (K3 - 1) * xp; e += blockDim.x) {
        const int k1 = fdiv(e, fxp), pp = e - k1 * xp, k = 1 + k1, j = j0 + pp;
        if (j < npair) {
            const Cx<T> zk = res[k * xp + pp], zm = res[(M3 - k) * xp + pp];
            Cx<T> *dst = zspec + ((size_t)k * Mt + y) * Mt + 2 * j;
            dst[0] = cx<T>((zk.re + zm.re) * (T)0.5, (zk.im - zm.im) * (T)0.5);
            if (2 * j + 1 < Mt) dst[1] = cx<T>((zk.im + zm.im) * (T)0.5, (zm.re - zk.re) * (T)0.5);
        }
    }
}

// ---- x forward: CTA = rb rows (slab s, y) of one class; smem [row][ns]
template <typename T, bool FROM_SLAB0>
__global__ void k_xfwd(int Mt, int ns, int kfirst, int nrows, FftDesc d, const Tw<T> *__restrict__ tw, int rb,
                       FastDiv frb, FastDiv fns, FastDiv fMt, const Cx<T> *__restrict__ zspec,
                       const double *__restrict__ slab0, Cx<T> *__restrict__ rows)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *b = a + (size_t)rb * ns;
    const int r0 = blockIdx.x * rb;
    for (int e = threadIdx.x; e < rb * ns; e += blockDim.x) {
        const int p = fdiv(e, fns), j = e - p * ns, r = r0 + p;
        Cx<T> v = cx<T>((T)0, (T)0);
        if (r < nrows && j < Mt) {
            const int s = fdiv(r, fMt), y = r - s * Mt;
            if (FROM_SLAB0) v = cx<T>((T)slab0[(size_t)y * Mt + j], (T)0);
            else v = zspec[((size_t)(kfirst + s) * Mt + y) * Mt + j];
        }
        a[e] = v;
    }
    __syncthreads();
    Cx<T> *res = fft_smem<T>(a, b, d, rb, frb, ns, 1, tw, -1);
    for (int e = threadIdx.x; e < rb * ns; e += blockDim.x) {
        const int p = fdiv(e, fns), r = r0 + p;
        if (r < nrows) rows[(size_t)r * ns + (e - p * ns)] = res[e];
    }
}

// ---- y pass with the scaling: CTA = (slab, chunk of xb columns); smem [y][p]
// Class 0 (k3 = 0) reads the FP64 symbol table, the other classes their own table
// of 4 pi / (ns^2 M3) exp(-(1-eta) kappa^2 / 4 xi^2 - (1-eta_z) k3^2 / 4 xi^2) / (kappa^2 + k3^2).
template <typename T, bool CLASS0>
__global__ void k_yscale(int Mt, int ns, int kfirst, int count, FftDesc d, const Tw<T> *__restrict__ tw, int xb,
                         FastDiv fxb, Cx<T> *__restrict__ rows, const double *__restrict__ sym0,
                         const T *__restrict__ symc)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *b = a + (size_t)ns * xb;
    const int nkc = (ns + xb - 1) / xb;
    const int s = blockIdx.x / nkc, kx0 = (blockIdx.x % nkc) * xb;
    Cx<T> *slab = rows + (size_t)s * Mt * ns;
    for (int e = threadIdx.x; e < ns * xb; e += blockDim.x) {
        const int y = fdiv(e, fxb), p = e - y * xb, kx = kx0 + p;
        a[e] = (y < Mt && kx < ns) ? slab[(size_t)y * ns + kx] : cx<T>((T)0, (T)0);
    }
    __syncthreads();
    Cx<T> *res = fft_smem<T>(a, b, d, xb, fxb, 1, xb, tw, -1);
    Cx<T> *oth = res == a ? b : a;
    for (int e = threadIdx.x; e < ns * xb; e += blockDim.x) {
        const int ky = fdiv(e, fxb), p = e - ky * xb, kx = kx0 + p;
        T S = (T)0;
        if (kx < ns) {
            if (CLASS0) S = (T)sym0[(size_t)ky * ns + kx];
            else S = symc[((size_t)s * ns + ky) * ns + kx];
        }
        res[e] = scale(res[e], S);
    }
    __syncthreads();
    res = fft_smem<T>(res, oth, d, xb, fxb, 1, xb, tw, +1);
    for (int e = threadIdx.x; e < Mt * xb; e += blockDim.x) {
        const int y = fdiv(e, fxb), p = e - y * xb, kx = kx0 + p;
        if (kx < ns) slab[(size_t)y * ns + kx] = res[e];
    }
}

// ---- x inverse: CTA = rb rows; inverse FFT along x, keep the first Mt points
template <typename T, bool TO_SLAB0>
__global__ void k_xinv(int Mt, int ns, int kfirst, int nrows, FftDesc d, const Tw<T> *__restrict__ tw, int rb,
                       FastDiv frb, FastDiv fns, FastDiv fMt, const Cx<T> *__restrict__ rows,
                       Cx<T> *__restrict__ zspec, double *__restrict__ slab0)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *b = a + (size_t)rb * ns;
    const int r0 = blockIdx.x * rb;
    for (int e = threadIdx.x; e < rb * ns; e += blockDim.x) {
        const int p = fdiv(e, fns), r = r0 + p;
        a[e] = r < nrows ? rows[(size_t)r * ns + (e - p * ns)] : cx<T>((T)0, (T)0);
    }
    __syncthreads();
    Cx<T> *res = fft_smem<T>(a, b, d, rb, frb, ns, 1, tw, +1);
    for (int e = threadIdx.x; e < rb * Mt; e += blockDim.x) {
        const int p = fdiv(e, fMt), x = e - p * Mt, r = r0 + p;
        if (r >= nrows) continue;
        const int s = fdiv(r, fMt), y = r - s * Mt;
        const Cx<T> v = res[p * ns + x];
        if (TO_SLAB0) slab0[(size_t)y * Mt + x] = (double)v.re;
        else zspec[((size_t)(kfirst + s) * Mt + y) * Mt + x] = v;
    }
}

// ---- z inverse on pencil pairs: Z = X_2j + i X_2j+1 over the Hermitian-completed spectra; the real and
// imaginary parts of its inverse FFT are the pencils 2j and 2j + 1 (for odd Mt the last pair has
// X_Mt = 0 and stores only its real part, so that the grid's padding stays exactly zero)
template <typename T>
__global__ void k_zinv_pair(int M3, int Mt, int K3, FftDesc d, const Tw<T> *__restrict__ tw, int xp, FastDiv fxp,
                            const Cx<T> *__restrict__ zspec, const double *__restrict__ slab0, T *__restrict__ grid)
{
    using V2 = typename Pair2<T>::type;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Cx<T> *a = reinterpret_cast<Cx<T> *>(smem_raw);
    Cx<T> *b = a + (size_t)M3 * xp;
    const int npair = (Mt + 1) / 2, nxc = (npair + xp - 1) / xp;
    const int y = blockIdx.x / nxc, j0 = (blockIdx.x % nxc) * xp;
    for (int e = threadIdx.x; e < M3 * xp; e += blockDim.x) {
        const int k = fdiv(e, fxp), pp = e - k * xp, j = j0 + pp;
        Cx<T> v = cx<T>((T)0, (T)0);
        if (j < npair) {
            const bool odd = 2 * j + 1 < Mt;  // the pair has its second pencil
            Cx<T> xe, xo = cx<T>((T)0, (T)0);
            if (k == 0) {
                xe = cx<T>((T)slab0[(size_t)y * Mt + 2 * j], (T)0);
                if (odd) xo = cx<T>((T)slab0[(size_t)y * Mt + 2 * j + 1], (T)0);
            } else if (k < K3) {
                const Cx<T> *src = zspec + ((size_t)k * Mt + y) * Mt + 2 * j;
                xe = src[0];
                if (odd) xo = src[1];
            } else {
                const Cx<T> *src = zspec + ((size_t)(M3 - k) * Mt + y) * Mt + 2 * j;
                xe = cx<T>(src[0].re, -src[0].im);
                if (odd) xo = cx<T>(src[1].re, -src[1].im);
            }
            v = cx<T>(xe.re - xo.im, xe.im + xo.re);
        }
        a[e] = v;
    }
    __syncthreads();
    Cx<T> *res = fft_smem<T>(a, b, d, xp, fxp, 1, xp, tw, +1);
    for (int e = threadIdx.x; e < M3 * xp; e += blockDim.x) {
        const int z = fdiv(e, fxp), pp = e - z * xp, j = j0 + pp;
        if (j < npair) {
            T *dst = grid + gidx(z, y, 2 * j, Mt, gnxb(Mt));
            if (2 * j + 1 < Mt) {
                V2 o;
                o.x = res[e].re;
                o.y = res[e].im;
                *reinterpret_cast<V2 *>(dst) = o;
            } else {
                dst[0] = res[e].re;
            }
        }
    }
}

// ---- k3 = 0 scaling table in FP64 (Eqs. 3.5, 3.9-3.10), including 1/(n0^2 M3)
__global__ void k_vico(int n0, double dkap, double R, double xi, double eta, double norm, double *__restrict__ sym)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n0 * n0) return;
    const int kx = i % n0, ky = i / n0;
    const double ax = dkap * signed_index(kx, n0), ay = dkap * signed_index(ky, n0);
    const double k2 = ax * ax + ay * ay;
    double G;
    if (k2 == 0.0) {
        G = R * R / 4.0 * (1.0 - 2.0 * log(R));
    } else {
        const double k = sqrt(k2);
        G = (1.0 - j0(R * k)) / k2 - R * log(R) * j1(R * k) / k;
    }
    sym[i] = norm * 4.0 * kPi * exp(-(1.0 - eta) * k2 / (4.0 * xi * xi)) * G;
}

// ---- k3 != 0 scaling tables (Eq. 3.5 with the Green's function of Eq. 3.6), one
// per class, computed in FP64 and rounded once per mode.  Built on the fly in FP32
// from per-axis factor tables, the symbol would carry those tables' roundings into
// every mode that shares an index, a bias of the FP32 grid energy that does not
// average out.
template <typename T>
__global__ void k_symbol(int ns, int count, int kfirst, double dkap, double dk3, double xi, double eta,
                         double etaz, double norm, T *__restrict__ sym)
{
    const size_t total = (size_t)count * ns * ns;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % ns), ky = (int)((i / ns) % ns), s = (int)(i / ((size_t)ns * ns));
        const double ax = dkap * signed_index(kx, ns), ay = dkap * signed_index(ky, ns);
        const double k3 = dk3 * (kfirst + s);
        const double kap2 = ax * ax + ay * ay;
        const double e = exp(-((1.0 - eta) * kap2 + (1.0 - etaz) * k3 * k3) / (4.0 * xi * xi));
        sym[i] = (T)(norm * e / (kap2 + k3 * k3));
    }
}

// ---- triply periodic k3 = 0 scaling table in FP64: 4 pi e^{-(1-eta) kappa^2/4xi^2} / kappa^2 for
// kappa != 0 and nothing at kappa = 0 (a neutral system in a conducting medium), including 1/(n^2 M3)
__global__ void k_k3zero_3p(int n, double dkap, double xi, double eta, double norm, double *__restrict__ sym)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * n) return;
    const double ax = dkap * signed_index(i % n, n), ay = dkap * signed_index(i / n, n);
    const double k2 = ax * ax + ay * ay;
    sym[i] = k2 == 0.0 ? 0.0 : norm * 4.0 * kPi * exp(-(1.0 - eta) * k2 / (4.0 * xi * xi)) / k2;
}

template <typename T> size_t cbytes() { return sizeof(Cx<T>); }

}  // namespace

void launch_k3zero_table_3p(se1p_plan *p, cudaStream_t s)
{
    const int n = p->n0;  // = M, the periodic grid
    const double dkap = 2.0 * kPi / (n * p->geo.h);
    const double norm = 1.0 / ((double)n * n * p->M3);
    k_k3zero_3p<<<(n * n + 255) / 256, 256, 0, s>>>(n, dkap, p->geo.xi, p->geo.eta, norm, p->b.sym0);
}

void launch_vico_table(se1p_plan *p, cudaStream_t s)
{
    const int n0 = p->n0;
    const double dkap = 2.0 * kPi / (n0 * p->geo.h);
    const double R = sqrt(2.0) * p->Mt * p->geo.h;
    const double norm = 1.0 / ((double)n0 * n0 * p->M3);
    k_vico<<<(n0 * n0 + 255) / 256, 256, 0, s>>>(n0, dkap, R, p->geo.xi, p->geo.eta, norm, p->b.sym0);
}

template <typename T> void launch_symbol_tables(se1p_plan *p, cudaStream_t s)
{
    const Geo &g = p->geo;
    for (int c = 1; c < 3; ++c) {
        const SlabClass &C = p->cls[c];
        if (C.count == 0) continue;
        const double dkap = 2.0 * kPi / (C.ns * g.h);
        const double dk3 = 2.0 * kPi / g.L[2];
        const double norm = 4.0 * kPi / ((double)p->M3 * C.ns * C.ns);
        const size_t total = (size_t)C.count * C.ns * C.ns;
        const int blocks = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
        k_symbol<T><<<blocks, 256, 0, s>>>(C.ns, C.count, C.kfirst, dkap, dk3, g.xi, g.eta, g.etaz, norm,
                                           (T *)C.sym);
    }
}
template void launch_symbol_tables<float>(se1p_plan *, cudaStream_t);
template void launch_symbol_tables<double>(se1p_plan *, cudaStream_t);

// Opt a kernel in to the device's largest dynamic shared memory (less its static shared memory).
template <typename K> cudaError_t allow_max_dynamic_smem(K kernel, int maxsm)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - (int)fa.sharedSizeBytes);
}

// Tensor map of the z forward pass over the x-blocked grid, a 4-D tensor [z][x / 8][y][x % 8] of T:
// boxes of min(2 xb, 8) x 1 x max(1, 2 xb / 8) x zbox values land in shared memory as [z][2 xb], the
// CTA's pencil pairs.  Used when the box's inner extent is a multiple of 16 bytes (every copied x
// offset within a block, 2 j0 mod 8, is then a multiple of 16 bytes too), 2 xb divides or is a multiple
// of the block, and zbox, the largest divisor of M3 up to 256 (the box limit per dimension), gives whole
// boxes.
template <typename T> void make_zfwd_tensor_map(se1p_plan *p)
{
    p->tma_zfwd = false;
    const int Mt = p->Mf, M3 = p->M3, xp = p->xb_z, nxb = gnxb(Mt);
    const int bx = 2 * xp < kXB ? 2 * xp : kXB, bxb = 2 * xp < kXB ? 1 : 2 * xp / kXB;
    if ((bx * sizeof(T)) % 16 != 0 || (2 * xp) % bx != 0 || bxb > 256) return;
    int zbox = 1;
    for (int v = 1; v <= 256 && v <= M3; ++v)
        if (M3 % v == 0) zbox = v;
    if (zbox < 8) return;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        return;
    }
    using Encode = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    const cuuint64_t dims[4] = {(cuuint64_t)kXB, (cuuint64_t)Mt, (cuuint64_t)nxb, (cuuint64_t)M3};
    const cuuint64_t strides[3] = {(cuuint64_t)kXB * sizeof(T), (cuuint64_t)Mt * kXB * sizeof(T),
                                   (cuuint64_t)nxb * Mt * kXB * sizeof(T)};
    const cuuint32_t box[4] = {(cuuint32_t)bx, 1u, (cuuint32_t)bxb, (cuuint32_t)zbox};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r = reinterpret_cast<Encode>(fn)(
        &p->tm_zfwd, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, p->b.gridf,
        dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return;
    p->tma_zfwd = true;
    p->tma_zbox = zbox;
}

template <typename T> int configure_fourier_kernels(se1p_plan *p)
{
    make_zfwd_tensor_map<T>(p);
    int dev;
    cudaGetDevice(&dev);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaSuccess;
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_zfwd_pair<T>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_zinv_pair<T>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_xfwd<T, false>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_xinv<T, false>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_yscale<T, false>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_xfwd<double, true>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_xinv<double, true>, maxsm));
    e = (cudaError_t)(e | allow_max_dynamic_smem(k_yscale<double, true>, maxsm));
    return e == cudaSuccess ? 0 : -1;
}

template <typename T> void launch_fourier(se1p_plan *p, cudaStream_t s)
{
    // the transformed grid's free-axis size (the extended grid itself for SE1P, the periodic grid
    // for triply periodic plans)
    const int Mt = p->Mf, M3 = p->M3, K3 = p->K3;
    // z forward
    {
        const int xb = p->xb_z;
        const size_t sm = 2 * (size_t)M3 * xb * cbytes<T>();
        const int nxc = ((Mt + 1) / 2 + xb - 1) / xb;  // xb pencil pairs per CTA
        k_zfwd_pair<T><<<Mt * nxc, 256, sm, s>>>(M3, Mt, K3, p->fd_z, (const Tw<T> *)p->b.tw_z, xb, make_fastdiv(xb),
                                                 (const T *)p->b.gridf, (Cx<T> *)p->b.zspec, p->b.slab0_in,
                                                 p->tm_zfwd, p->tma_zfwd ? 1 : 0, p->tma_zbox, p->b.status,
                                                 p->spin_limit);
    }
    // the three slab classes are independent between the z passes: classes 0 (k3 = 0, FP64)
    // and 1 (set I) run on the plan's two Fourier streams, class 2 (set J) on s
    cudaEventRecord(p->ev_f[0], s);
    cudaStreamWaitEvent(p->s_f[0], p->ev_f[0], 0);
    cudaStreamWaitEvent(p->s_f[1], p->ev_f[0], 0);
    const cudaStream_t s_main = s;
    const FastDiv fMt = make_fastdiv(Mt);
    for (int c = 0; c < 3; ++c) {
        const SlabClass &C = p->cls[c];
        if (C.count == 0) continue;
        const cudaStream_t s = c == 2 ? s_main : p->s_f[c];  // this class's stream
        const int nrows = C.count * Mt;
        const FastDiv frb = make_fastdiv(C.rb), fns = make_fastdiv(C.ns), fxb = make_fastdiv(C.xb);
        if (c == 0) {
            const size_t smx = 2 * (size_t)C.rb * C.ns * cbytes<double>();
            k_xfwd<double, true><<<(nrows + C.rb - 1) / C.rb, 256, smx, s>>>(
                Mt, C.ns, 0, nrows, C.fd, (const Tw<double> *)C.tw, C.rb, frb, fns, fMt, nullptr, p->b.slab0_in,
                (Cx<double> *)C.rows);
            const int nkc = (C.ns + C.xb - 1) / C.xb;
            const size_t smy = 2 * (size_t)C.ns * C.xb * cbytes<double>();
            k_yscale<double, true><<<C.count * nkc, 256, smy, s>>>(Mt, C.ns, 0, C.count, C.fd, (const Tw<double> *)C.tw,
                                                                  C.xb, fxb, (Cx<double> *)C.rows, p->b.sym0, nullptr);
            k_xinv<double, true><<<(nrows + C.rb - 1) / C.rb, 256, smx, s>>>(
                Mt, C.ns, 0, nrows, C.fd, (const Tw<double> *)C.tw, C.rb, frb, fns, fMt, (const Cx<double> *)C.rows,
                nullptr, p->b.slab0_out);
        } else {
            const size_t smx = 2 * (size_t)C.rb * C.ns * cbytes<T>();
            k_xfwd<T, false><<<(nrows + C.rb - 1) / C.rb, 256, smx, s>>>(
                Mt, C.ns, C.kfirst, nrows, C.fd, (const Tw<T> *)C.tw, C.rb, frb, fns, fMt, (const Cx<T> *)p->b.zspec,
                nullptr, (Cx<T> *)C.rows);
            const int nkc = (C.ns + C.xb - 1) / C.xb;
            const size_t smy = 2 * (size_t)C.ns * C.xb * cbytes<T>();
            k_yscale<T, false><<<C.count * nkc, 256, smy, s>>>(Mt, C.ns, C.kfirst, C.count, C.fd, (const Tw<T> *)C.tw,
                                                              C.xb, fxb, (Cx<T> *)C.rows, nullptr, (const T *)C.sym);
            k_xinv<T, false><<<(nrows + C.rb - 1) / C.rb, 256, smx, s>>>(
                Mt, C.ns, C.kfirst, nrows, C.fd, (const Tw<T> *)C.tw, C.rb, frb, fns, fMt, (const Cx<T> *)C.rows,
                (Cx<T> *)p->b.zspec, nullptr);
        }
    }
    cudaEventRecord(p->ev_f[1], p->s_f[0]);
    cudaEventRecord(p->ev_f[2], p->s_f[1]);
    cudaStreamWaitEvent(s, p->ev_f[1], 0);
    cudaStreamWaitEvent(s, p->ev_f[2], 0);
    // z inverse
    {
        const int xb = p->xb_z;
        const size_t sm = 2 * (size_t)M3 * xb * cbytes<T>();
        const int nxc = ((Mt + 1) / 2 + xb - 1) / xb;
        k_zinv_pair<T><<<Mt * nxc, 256, sm, s>>>(M3, Mt, K3, p->fd_z, (const Tw<T> *)p->b.tw_z, xb, make_fastdiv(xb),
                                                 (const Cx<T> *)p->b.zspec, p->b.slab0_out, (T *)p->b.gridf);
    }
}

template void launch_fourier<float>(se1p_plan *, cudaStream_t);
template void launch_fourier<double>(se1p_plan *, cudaStream_t);
template int configure_fourier_kernels<float>(se1p_plan *);
template int configure_fourier_kernels<double>(se1p_plan *);

}  // namespace se1p
