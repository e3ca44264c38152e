// Internal declarations shared by the translation units of libse1p.
//
// Grid layout (all precisions): real grids are [z][y][x] with x fastest,
// M3 x Mt x Mt points; the free-axis origin is at -P h/2 (a particle at x sits
// at x + P h/2 on [0, Mt h)), z is periodic with M3 points.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "se1p.h"

namespace se1p {

// ------------------------------------------------------------------ status bits
enum : int {
    FLAG_OUT_OF_BOX = 1,
    FLAG_NAN = 2,
    FLAG_NOT_NEUTRAL = 4,
    FLAG_CAPACITY = 8,
    FLAG_TIMEOUT = 16,
};

constexpr double kPi = 3.14159265358979323846264338327950288;

// multi-block scan of the cell counts: 4096 counts per block, at most kScanTmp blocks (2^22 cells)
constexpr int kScanChunk = 4096;
constexpr int kScanTmp = (1 << 22) / kScanChunk + 2;

// ------------------------------------------------------------------ complex
template <typename T> struct Cx;
template <> struct __align__(8) Cx<float> { float re, im; };
template <> struct __align__(16) Cx<double> { double re, im; };

// Two FP32 values in one 64-bit register.  The .f32x2 instructions of sm_100 and later do
// two round-to-nearest FP32 operations per issued instruction, with the results of the two
// scalar operations; they halve the issue slots of FP32 arithmetic on independent pairs.
using f32x2 = unsigned long long;
__device__ __forceinline__ f32x2 f2_pack(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 f2_splat(float v) { return f2_pack(v, v); }
__device__ __forceinline__ float2 f2_unpack(f32x2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f32x2 f2_add(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_mul(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c)  // a b + c
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <typename T> __device__ __forceinline__ Cx<T> cx(T re, T im) { Cx<T> r; r.re = re; r.im = im; return r; }
template <typename T> __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return cx<T>(a.re + b.re, a.im + b.im); }
template <typename T> __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return cx<T>(a.re - b.re, a.im - b.im); }
template <typename T> __device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b)
{
    return cx<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// multiply by s*i, s = +-1
template <typename T> __device__ __forceinline__ Cx<T> mul_si(Cx<T> a, int s)
{
    return s > 0 ? cx<T>(-a.im, a.re) : cx<T>(a.im, -a.re);
}
template <typename T> __device__ __forceinline__ Cx<T> scale(Cx<T> a, T s) { return cx<T>(a.re * s, a.im * s); }

// Butterfly constants c (cosines and sines of 2 pi m / R) as an exact double.  In FP32,
// c is applied as hi + lo, so each product is rounded once from a nearly exact value:
// a constant rounded to float would scale every butterfly output alike, a bias of the
// transform's gain that does not average out (it shows in the energy, where the
// self-interaction through the grid cancels against the self term).  FP64 uses c.
template <typename T> __device__ __forceinline__ T mul_c(T v, double c)
{
    if constexpr (sizeof(T) == sizeof(double)) {
        return v * c;
    } else {
        const float hi = (float)c, lo = (float)(c - (double)hi);
        return fmaf(v, hi, v * lo);
    }
}
// acc + v * c with c as above
template <typename T> __device__ __forceinline__ T fma_c(T v, double c, T acc)
{
    if constexpr (sizeof(T) == sizeof(double)) {
        return fma(v, c, acc);
    } else {
        const float hi = (float)c, lo = (float)(c - (double)hi);
        return fmaf(v, hi, fmaf(v, lo, acc));
    }
}

// Twiddle factor w^t = exp(-2 pi i t / n).  In FP32 each component is kept as hi + lo:
// rounded alone, the few roots of unity that a whole pass uses (an early pass uses
// only the 64th roots) have magnitudes that are off in the same direction, which
// scales the transform by ~1 - 3e-8 and biases the grid energy.
template <typename T> struct Tw;
template <> struct __align__(16) Tw<float> { float re, im, lre, lim; };
template <> struct __align__(16) Tw<double> { double re, im; };

// v * w (s < 0, forward) or v * conj(w) (s > 0, inverse); FP32 adds the lo products first
template <typename T> __device__ __forceinline__ Cx<T> tw_mul(Cx<T> v, Tw<T> w, int s)
{
    const T wi = s > 0 ? -w.im : w.im;
    if constexpr (sizeof(T) == sizeof(double)) {
        return cx<T>(v.re * w.re - v.im * wi, v.re * wi + v.im * w.re);
    } else {
        const float li = s > 0 ? -w.lim : w.lim;
        const float re = fmaf(v.re, w.re, fmaf(-v.im, wi, fmaf(v.re, w.lre, -v.im * li)));
        const float im = fmaf(v.re, wi, fmaf(v.im, w.re, fmaf(v.re, li, v.im * w.lre)));
        return cx<float>(re, im);
    }
}

// ------------------------------------------------------------------ bulk tensor copies (TMA)
// One CTA-local mbarrier tracks the bytes of the tensor copies a CTA issues; every wait on it is
// bounded by an iteration count, after which the caller records FLAG_TIMEOUT and drains.
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor-copy unit
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// true when the phase completed within `limit` polls (each poll may suspend the thread briefly)
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned phase, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}
// 4-D tiled copy global -> shared of the box at (c0, c1, c2, c3) of tensor map `tm`, completing on `bar`
__device__ __forceinline__ void tma_load_4d(unsigned dst, const void *tm, int c0, int c1, int c2, int c3, unsigned bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}
constexpr long long kDrainPolls = 1ll << 24;  // bound of the wait for copies still in flight after a timeout

// ------------------------------------------------------------------ FFT descriptor
// A length-n transform factored into radices (applied first to last).  The
// twiddle table holds w^t = exp(-2 pi i t / n), t = 0..n-1.
// Exact floor(x / d) for 0 <= x < 2^31 and 1 <= d < 2^31 with one multiply-high, an add and a
// shift: the round-up method of Granlund and Montgomery (Division by invariant integers using
// multiplication, PLDI 1994), l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (umulhi(m, x) + x) >> l.  Built on the host for divisors known at plan creation, so that
// index arithmetic in the hot loops avoids the integer division sequence.
struct FastDiv {
    unsigned d = 1, m = 1, l = 0;
};
inline FastDiv make_fastdiv(unsigned d)
{
    FastDiv f;
    f.d = d;
    f.l = 0;
    while ((1ull << f.l) < d) ++f.l;
    f.m = (unsigned)(((1ull << 32) * ((1ull << f.l) - d)) / d + 1);
    return f;
}
__device__ __forceinline__ int fdiv(int x, const FastDiv &f)
{
    return (int)((__umulhi((unsigned)x, f.m) + (unsigned)x) >> f.l);
}

// Mixed-radix plan of one FFT length: radices in pass order, and per pass the dividers of the
// butterfly span Ns (product of the earlier radices) and of the butterfly count n / R.
struct FftDesc {
    int n;
    int nrad;
    int rad[24];
    FastDiv ns[24], nb[24];
};

// Small DFTs, X_k = sum_j a_j exp(s 2 pi i j k / R), s = -1 forward, +1 inverse.
template <typename T> __device__ __forceinline__ void dft2(Cx<T> *v)
{
    Cx<T> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
}

template <typename T> __device__ __forceinline__ void dft4(Cx<T> *v, int s)
{
    Cx<T> t0 = v[0] + v[2], t1 = v[0] - v[2], t2 = v[1] + v[3], t3 = v[1] - v[3];
    v[0] = t0 + t2;
    v[2] = t0 - t2;
    Cx<T> r = mul_si(t3, s);
    v[1] = t1 + r;
    v[3] = t1 - r;
}

template <typename T> __device__ __forceinline__ void dft8(Cx<T> *v, int s)
{
    Cx<T> e[4] = {v[0], v[2], v[4], v[6]};
    Cx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e, s);
    dft4(o, s);
    // w8^k = exp(s 2 pi i k / 8) = (+-1 + s i) / sqrt(2) for k = 1, 3:
    // o w8 = ((+-a - s b) + i (+-b + s a)) / sqrt(2) for o = a + i b
    constexpr double r = 0.70710678118654752440;
    const T sa1 = s * o[1].re, sb1 = s * o[1].im, sa3 = s * o[3].re, sb3 = s * o[3].im;
    const Cx<T> o1 = cx<T>(mul_c<T>(o[1].re - sb1, r), mul_c<T>(o[1].im + sa1, r));
    const Cx<T> o3 = cx<T>(mul_c<T>(-o[3].re - sb3, r), mul_c<T>(-o[3].im + sa3, r));
    const Cx<T> o2 = mul_si(o[2], s);
    v[0] = e[0] + o[0];
    v[4] = e[0] - o[0];
    v[1] = e[1] + o1;
    v[5] = e[1] - o1;
    v[2] = e[2] + o2;
    v[6] = e[2] - o2;
    v[3] = e[3] + o3;
    v[7] = e[3] - o3;
}

// Odd radix by symmetric pairs: X_k = a0 + sum_{j=1}^{(R-1)/2} [(a_j + a_{R-j}) c_{jk}
//                                      + s i (a_j - a_{R-j}) s_{jk}],  c_m = cos(2 pi m/R).
template <typename T, int R> __device__ __forceinline__ void dft_odd(Cx<T> *v, int s)
{
    constexpr int H = (R - 1) / 2;
    double c[R], sn[R];
    if constexpr (R == 3) {
        const double cc[3] = {1, -0.5, -0.5};
        const double ss[3] = {0, 0.86602540378443864676, -0.86602540378443864676};
        for (int m = 0; m < R; ++m) { c[m] = cc[m]; sn[m] = ss[m]; }
    } else if constexpr (R == 5) {
        const double cc[5] = {1, 0.30901699437494742410, -0.80901699437494742410, -0.80901699437494742410,
                              0.30901699437494742410};
        const double ss[5] = {0, 0.95105651629515357212, 0.58778525229247312917, -0.58778525229247312917,
                              -0.95105651629515357212};
        for (int m = 0; m < R; ++m) { c[m] = cc[m]; sn[m] = ss[m]; }
    } else {
        const double cc[7] = {1, 0.62348980185873353053, -0.22252093395631440429, -0.90096886790241912624,
                              -0.90096886790241912624, -0.22252093395631440429, 0.62348980185873353053};
        const double ss[7] = {0, 0.78183148246802980871, 0.97492791218182360702, 0.43388373911755812048,
                              -0.43388373911755812048, -0.97492791218182360702, -0.78183148246802980871};
        for (int m = 0; m < R; ++m) { c[m] = cc[m]; sn[m] = ss[m]; }
    }
    Cx<T> sp[H], sm[H];
    Cx<T> x0 = v[0];
    Cx<T> tot = x0;
#pragma unroll
    for (int j = 1; j <= H; ++j) {
        sp[j - 1] = v[j] + v[R - j];
        sm[j - 1] = v[j] - v[R - j];
        tot = tot + sp[j - 1];
    }
    v[0] = tot;
#pragma unroll
    for (int k = 1; k < R; ++k) {
        Cx<T> acc = x0;
        Cx<T> accs = cx<T>(0, 0);
#pragma unroll
        for (int j = 1; j <= H; ++j) {
            const int m = (j * k) % R;
            acc = cx<T>(fma_c<T>(sp[j - 1].re, c[m], acc.re), fma_c<T>(sp[j - 1].im, c[m], acc.im));
            accs = cx<T>(fma_c<T>(sm[j - 1].re, sn[m], accs.re), fma_c<T>(sm[j - 1].im, sn[m], accs.im));
        }
        v[k] = acc + mul_si(accs, s);
    }
}

// One Stockham pass of radix R over `npen` pencils of length n held in shared
// memory: element j of pencil p lives at buf[p * sp + j * sj].
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const Cx<T> *__restrict__ src, Cx<T> *__restrict__ dst, int n,
                                              int Ns, const FastDiv &fns, const FastDiv &fnb, const FastDiv &fpen,
                                              int npen, int sp, int sj, const Tw<T> *__restrict__ tw, int s)
{
    const int nb = n / R;
    const int total = nb * npen;
    const int twmul = n / (Ns * R);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int i, p;
        if (sj == 1) {
            p = fdiv(idx, fnb);
            i = idx - p * nb;
        } else {
            i = fdiv(idx, fpen);
            p = idx - i * npen;
        }
        const int q = fdiv(i, fns), k = i - q * Ns;
        Cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[p * sp + (i + r * nb) * sj];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = tw_mul(v[r], tw[r * k * twmul], s);
        }
        if constexpr (R == 2) dft2(v);
        else if constexpr (R == 4) dft4(v, s);
        else if constexpr (R == 8) dft8(v, s);
        else dft_odd<T, R>(v, s);
        const int base = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[p * sp + (base + r * Ns) * sj] = v[r];
    }
}

// Batched in-shared-memory FFT (unnormalised; s = -1 forward, +1 inverse).
// a holds the input, b is scratch of the same shape; returns the buffer that
// holds the result.  Must be called by all threads of the block.  fpen divides by npen.
template <typename T>
__device__ Cx<T> *fft_smem(Cx<T> *a, Cx<T> *b, const FftDesc &d, int npen, const FastDiv &fpen, int sp, int sj,
                           const Tw<T> *__restrict__ tw, int s)
{
    int Ns = 1;
    for (int st = 0; st < d.nrad; ++st) {
        const int R = d.rad[st];
        const FastDiv &fns = d.ns[st], &fnb = d.nb[st];
        switch (R) {
        case 2: stockham_pass<T, 2>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        case 3: stockham_pass<T, 3>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        case 4: stockham_pass<T, 4>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        case 5: stockham_pass<T, 5>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        case 7: stockham_pass<T, 7>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        default: stockham_pass<T, 8>(a, b, d.n, Ns, fns, fnb, fpen, npen, sp, sj, tw, s); break;
        }
        __syncthreads();
        Cx<T> *t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// ------------------------------------------------------------------ particles

// e^x in FP32 for the window exponents, x in [-87, 0]: e^x = 2^n e^r with
// n = rint(x / ln 2) and r = x - n ln 2 (Cody and Waite's reduction: ln 2 in two
// parts, the first with 8 trailing zero bits so that n * hi is exact for |n| < 256),
// e^r by its Taylor series to r^8 (|r| <= ln 2 / 2, truncation < 3e-10), 2^n exact.
// Every step rounds to nearest, so the result (within ~1.2 ulp) has no systematic
// bias, which a window value must not have: the FP32 grid's self-interaction of
// each charge would carry it into the energy.
__host__ __device__ __forceinline__ float exp_window(float x)
{
    x = fmaxf(x, -87.0f);  // keeps 2^n normal; e^-87 ~ 1.6e-38 is below any window value used
    const float n = rintf(x * 1.44269504088896341f);
    float r = fmaf(n, -0.693145751953125f, x);
    r = fmaf(n, -1.42860677e-06f, r);
    float p = 2.48015873e-05f;  // 1/8!
    p = fmaf(p, r, 1.98412698e-04f);
    p = fmaf(p, r, 1.38888889e-03f);
    p = fmaf(p, r, 8.33333333e-03f);
    p = fmaf(p, r, 4.16666667e-02f);
    p = fmaf(p, r, 1.66666667e-01f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    const int bits = ((int)n + 127) << 23;  // 2^n
#ifdef __CUDA_ARCH__
    return p * __int_as_float(bits);
#else
    float two_n;
    memcpy(&two_n, &bits, sizeof(two_n));
    return p * two_n;
#endif
}


// Particle record in spread-bin order.  t_a = (coordinate from grid origin)/h_a;
// i0 is the first support index (free axes in [0, Mt-P], z wrapped into [0, M3));
// g = t - i0 - c with c = P/2 (even P) or (P-1)/2 (odd P), so grid point
// i0 + j lies at distance (g - (j - c)) h from the particle.
template <typename T> struct PartRec {
    int i0[3];
    int orig;
    T g[3];
    T q;
};

// Real-space record in cell order: absolute coordinates, computed in FP64 and
// stored as an unevaluated sum hi + lo of two T values (lo = 0 for T = double),
// charge and caller index.  With FP32 the split keeps pair displacements
// accurate to a few ulps of |d| instead of a few ulps of the coordinates.
template <typename T> struct __align__(sizeof(T) == 4 ? 16 : 32) CellRec {
    T xh, yh, zh, q;
    T xl, yl, zl;
    int orig;
};

// FP64 factors applied to a gather's FP32 sums (potential; force in x, y; force in z).
struct GatherScale {
    double phi, fxy, fz;
};

// Geometry passed by value to kernels.
struct Geo {
    int M3, Mt, P, K3;
    int c;            // support centre offset (P/2 or (P-1)/2)
    int nbx, nby, nbz, nbins;  // spread bins over support-start indices
    int ncx, ncy, ncz, ncells; // real-space cells
    double L[3];
    double h, hz, off;         // spacings, free-axis grid origin shift P h / 2
    double inv_h, inv_hz;      // 1/h, 1/hz
    double xi, eta, etaz;
    double wnorm_xy, wnorm_z;  // (2 xi^2 / (pi eta))^{1/2} per axis
    double alpha_xy, alpha_z;  // 2 xi^2 h^2 / eta per axis (exponent scale in grid units)
    double cs[3];              // cell sizes
    double rc, rc2;
    int nIm;                   // number of k3 > 0 modes in the set I
    int per3;                  // 1: x and y periodic too (the SE3P comparison method), 0: free (SE1P)
};

constexpr int kBin = 8;  // spread bin / tile edge in grid points

// Storage of the real grids (the gridding output, the transformed grid, and the periodic grid of
// triply periodic plans): x-blocks of kXB points, [z][x / kXB][y][x % kXB], with n x n points per
// z plane stored as gnxb(n) blocks of n rows.  The rows of one block are kXB values apart, so the
// kXB x-points of consecutive y rows are contiguous: a warp reading a particle's support touches
// whole 128-byte lines (four FP32 rows per line) instead of one or two lines per row.  x points
// from n up to the end of the last block are padding and hold zeros.
constexpr int kXB = 8;
__host__ __device__ __forceinline__ int gnxb(int n) { return (n + kXB - 1) / kXB; }
__host__ __device__ __forceinline__ size_t gidx(int z, int y, int x, int n, int nxb)
{
    return (((size_t)z * nxb + (x >> 3)) * n + y) * kXB + (x & (kXB - 1));
}
__host__ __device__ __forceinline__ size_t grid_points(int M3, int n) { return (size_t)M3 * gnxb(n) * n * kXB; }

}  // namespace se1p
