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
template <> __device__ __forceinline__ float exp_t<float>(float v) { return exp2f(v * 1.4426950408889634f); }
template <> __device__ __forceinline__ double exp_t<double>(double v) { return exp(v); }

constexpr int kRealWarps = 4;  // warps per CTA (warps work independently)
constexpr int kRealSplit = 4;  // warps sharing one group of 32 targets (source rows split between them)
constexpr int kCand = 96;      // per-warp candidate list (flushed at >= 64)

template <typename T> __device__ __forceinline__ T rsqrt_t(T v);
// 1/sqrt with one Newton step after the hardware estimate, so that r = r2 / sqrt(r2)
// is within ~1 ulp (erfc(xi r) near rc amplifies the relative error of r ~10x).
template <> __device__ __forceinline__ float rsqrt_t<float>(float v)
{
    const float y = rsqrtf(v);
    return y * fmaf(-0.5f * v * y, y, 1.5f);
}
template <> __device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }

// FP32 erfc(x) given E = exp(-x^2): erfc = E * erfcx(x), erfcx(x) ~ t * poly(t - tc),
// t = 1/(1 + p x), fitted on x in [0, 7] by gen_erfcx_fit.py (fit error 1.8e-8,
// FP32 evaluation 3.3e-7 relative).  Branch-free; shares E with the force term.
constexpr float kErfcxP = 0.5f, kErfcxTc = 6.111111111e-01f;
__device__ __forceinline__ float erfc_from_exp(float x, float E)
{
    const float c[11] = {5.942152530e-01f, 8.157567363e-01f, 5.936057846e-01f, 5.940804148e-02f,
                         -2.097116850e-01f, -3.031409504e-02f, 1.127779386e-01f, -1.429198095e-02f,
                         -6.719807144e-02f, 2.960473828e-02f, 3.436364278e-02f};
    const float d = fmaf(kErfcxP, x, 1.0f);
    float t = __fdividef(1.0f, d);
    t = t * fmaf(-d, t, 2.0f);  // one Newton step on the hardware reciprocal
    const float u = t - kErfcxTc;
    // Estrin's scheme: dependency depth 4 instead of 10 for Horner
    const float u2 = u * u, u4 = u2 * u2, u8 = u4 * u4;
    const float p01 = fmaf(c[1], u, c[0]), p23 = fmaf(c[3], u, c[2]), p45 = fmaf(c[5], u, c[4]);
    const float p67 = fmaf(c[7], u, c[6]), p89 = fmaf(c[9], u, c[8]);
    const float q03 = fmaf(p23, u2, p01), q47 = fmaf(p67, u2, p45), q8a = fmaf(c[10], u2, p89);
    const float acc = fmaf(q8a, u8, fmaf(q47, u4, q03));
    return E * (acc * t);
}
__device__ __forceinline__ double erfc_from_exp(double x, double) { return erfc(x); }

// z displacement of target m from a source image shifted by sh (a multiple of L3).
// The shift is applied first to whichever coordinate lies at the far wall, so the
// large cancellation (z close to +-L3) is exact (Sterbenz) and only the final,
// small difference is rounded; lo parts then restore the FP64 coordinates.
template <typename T> __device__ __forceinline__ T image_dz(T zm, T zs, T sh)
{
    return sh > (T)0 ? (zm - sh) - zs : (sh < (T)0 ? zm - (zs + sh) : zm - zs);
}

// Real-space sum, warp-centric.  Warp w owns the 32 consecutive targets
// 32w..32w+31 in cell order (all lanes busy, any cell boundaries), so its
// targets occupy a small box of cells.  Sources come from that box expanded by
// S = ceil(rc / cell edge) cells per axis; for each (y, z) cell row the x-range
// is contiguous in cell order, i.e. one source range; z images come from
// unwrapped rows nz_u = nz + wrap * ncz, shifted by wrap * L3.
//
// Sources are read 32 at a time, one per lane, and tested in parallel against
// the warp's target bounding box grown by rc; the survivors are compacted by
// ballot into a per-warp list.  When the list holds >= 32 candidates every lane
// marks (cheap hi-part test, threshold widened by 1e-5) the candidates within rc
// of its own target, then walks its marks: exact displacement (hi + lo, shift
// hi + lo), exact r <= rc test, erfc and exp.
template <typename T>
__global__ void __launch_bounds__(32 * kRealWarps) k_real(Geo g, int n, const int *__restrict__ cell_start,
                                                          const CellRec<T> *__restrict__ cells,
                                                          const int *__restrict__ cell_key,
                                                          double *__restrict__ phi, double *__restrict__ frc,
                                                          int accumulate)
{
    __shared__ CellRec<T> cand[kRealWarps][kCand];
    __shared__ float4 cpos[kRealWarps][kCand];  // phase-1 copy: x, y, z + shift (float), q
    __shared__ T cshh[kRealWarps][kCand], cshl[kRealWarps][kCand];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kRealWarps + wib;
    const int warp = gw / kRealSplit, part = gw % kRealSplit;  // target group, share of the source rows
    const int t = warp * 32 + lane;
    if (warp * 32 >= n) return;  // whole warp beyond the particles
    const bool valid = t < n;
    CellRec<T> me;
    int cx = 0, cy = 0, cz = 0;
    if (valid) {
        me = cells[t];
        const int cell = cell_key[me.orig];
        cx = cell % g.ncx;
        cy = (cell / g.ncx) % g.ncy;
        cz = cell / (g.ncx * g.ncy);
    } else {
        me.xh = me.yh = me.zh = me.q = me.xl = me.yl = me.zl = (T)0;
        me.orig = -1;
    }
    const unsigned full = 0xffffffffu;
    const int big = 1 << 30;
    // box of the warp's target cells (invalid lanes do not widen it)
    const int cx0 = __reduce_min_sync(full, valid ? cx : big), cx1 = __reduce_max_sync(full, valid ? cx : -big);
    const int cy0 = __reduce_min_sync(full, valid ? cy : big), cy1 = __reduce_max_sync(full, valid ? cy : -big);
    const int cz0 = __reduce_min_sync(full, valid ? cz : big), cz1 = __reduce_max_sync(full, valid ? cz : -big);
    // bounding box of the warp's target positions (coordinates >= 0: float bits order like ints)
    const float fx = (float)me.xh, fy = (float)me.yh, fz = (float)me.zh;
    const float bx0 = __int_as_float(__reduce_min_sync(full, valid ? __float_as_int(fx) : 0x7f7fffff));
    const float bx1 = __int_as_float(__reduce_max_sync(full, valid ? __float_as_int(fx) : 0));
    const float by0 = __int_as_float(__reduce_min_sync(full, valid ? __float_as_int(fy) : 0x7f7fffff));
    const float by1 = __int_as_float(__reduce_max_sync(full, valid ? __float_as_int(fy) : 0));
    const float bz0 = __int_as_float(__reduce_min_sync(full, valid ? __float_as_int(fz) : 0x7f7fffff));
    const float bz1 = __int_as_float(__reduce_max_sync(full, valid ? __float_as_int(fz) : 0));
    const float rbox = (float)(g.rc + 1e-5 * (g.L[0] + g.L[1] + g.L[2]));
    const float rbox2 = rbox * rbox;
    const int Sx = (int)ceil(g.rc / g.cs[0] - 1e-9), Sy = (int)ceil(g.rc / g.cs[1] - 1e-9),
              Sz = (int)ceil(g.rc / g.cs[2] - 1e-9);
    const int nx_lo = max(cx0 - Sx, 0), nx_hi = min(cx1 + Sx, g.ncx - 1);
    const int ny_lo = max(cy0 - Sy, 0), ny_hi = min(cy1 + Sy, g.ncy - 1);
    const T xi = (T)g.xi, rc2 = (T)g.rc2;
    const T two_xi_sqpi = (T)(2.0 * g.xi / sqrt(kPi));
    const T xi2 = (T)(g.xi * g.xi);
    CellRec<T> *cl = cand[wib];
    T *ch = cshh[wib], *cll = cshl[wib];
    const unsigned lt_mask = (1u << lane) - 1u;
    double aphi = 0, afx = 0, afy = 0, afz = 0;
    int ncand = 0;

    float4 *cp = cpos[wib];
    const float mxf = (float)me.xh, myf = (float)me.yh, mzf = (float)me.zh;
    // phase-1 threshold: rc widened by 1e-5 rc plus a few float ulps of the box size, so the
    // float test (coordinates and image shift rounded to float) never drops a true pair
    const double lmax = fmax(fmax(g.L[0], g.L[1]), g.L[2]);
    const float rc2wf = (float)((g.rc * (1.0 + 1e-5) + 5e-7 * lmax) * (g.rc * (1.0 + 1e-5) + 5e-7 * lmax));

    auto process = [&](int nc) {
        __syncwarp();
        // phase 1: candidates within rc of this lane's target (float test, widened threshold)
        unsigned m0 = 0u, m1 = 0u, m2 = 0u;
        if (valid) {
            const int n0 = min(nc, 32), n1 = min(nc, 64);
            for (int j = 0; j < n0; ++j) {
                const float4 c = cp[j];
                const float dx = mxf - c.x, dy = myf - c.y, dz = mzf - c.z;
                if (dx * dx + dy * dy + dz * dz <= rc2wf) m0 |= 1u << j;
            }
            for (int j = 32; j < n1; ++j) {
                const float4 c = cp[j];
                const float dx = mxf - c.x, dy = myf - c.y, dz = mzf - c.z;
                if (dx * dx + dy * dy + dz * dz <= rc2wf) m1 |= 1u << (j - 32);
            }
            for (int j = 64; j < nc; ++j) {
                const float4 c = cp[j];
                const float dx = mxf - c.x, dy = myf - c.y, dz = mzf - c.z;
                if (dx * dx + dy * dy + dz * dz <= rc2wf) m2 |= 1u << (j - 64);
            }
        }
        // phase 2: exact displacement and the pair terms, each lane walking its own marks
        T pphi = 0, pfx = 0, pfy = 0, pfz = 0;
        while (m0 | m1 | m2) {
            int j;
            if (m0) {
                j = __ffs(m0) - 1;
                m0 &= m0 - 1u;
            } else if (m1) {
                j = 32 + __ffs(m1) - 1;
                m1 &= m1 - 1u;
            } else {
                j = 64 + __ffs(m2) - 1;
                m2 &= m2 - 1u;
            }
            const CellRec<T> sr = cl[j];
            const T sh = ch[j];
            if (sr.orig == me.orig && sh == (T)0) continue;  // the target itself
            T dx = me.xh - sr.xh, dy = me.yh - sr.yh, dz = image_dz(me.zh, sr.zh, sh);
            if constexpr (sizeof(T) < sizeof(double)) {
                dx += me.xl - sr.xl;
                dy += me.yl - sr.yl;
                dz += (me.zl - sr.zl) - cll[j];
            }
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > rc2) continue;
            const T rinv = rsqrt_t<T>(r2);
            const T r = r2 * rinv;
            const T E = exp_t<T>(-xi2 * r2);
            const T e = erfc_from_exp(xi * r, E) * rinv;
            pphi += sr.q * e;
            const T fs = sr.q * (two_xi_sqpi * E + e) * rinv * rinv;
            pfx += fs * dx;
            pfy += fs * dy;
            pfz += fs * dz;
        }
        aphi += (double)pphi;
        afx += (double)pfx;
        afy += (double)pfy;
        afz += (double)pfz;
        __syncwarp();
    };

    const int nyr = ny_hi - ny_lo + 1;
    const int nrows = (cz1 + Sz - (cz0 - Sz) + 1) * max(nyr, 0);
    for (int rr = part; rr < nrows; rr += kRealSplit) {
        const int nzu = cz0 - Sz + rr / nyr, ny = ny_lo + rr % nyr;
        const int wrap = nzu >= 0 ? nzu / g.ncz : -((-nzu + g.ncz - 1) / g.ncz);
        const int nz = nzu - wrap * g.ncz;
        const double shd = wrap * g.L[2];
        const T sh = (T)shd, shl = (T)(shd - (double)sh);
        const float shf = (float)shd;
        {
            const int row = (nz * g.ncy + ny) * g.ncx;
            const int sbeg = cell_start[row + nx_lo], send = cell_start[row + nx_hi + 1];
            for (int s0 = sbeg; s0 < send; s0 += 32) {
                const int si = s0 + lane;
                bool keep = false;
                CellRec<T> rec;
                if (si < send) {
                    rec = cells[si];
                    const float sx = (float)rec.xh, sy = (float)rec.yh, sz = (float)rec.zh + shf;
                    const float ex = fmaxf(fmaxf(bx0 - sx, sx - bx1), 0.0f);
                    const float ey = fmaxf(fmaxf(by0 - sy, sy - by1), 0.0f);
                    const float ez = fmaxf(fmaxf(bz0 - sz, sz - bz1), 0.0f);
                    keep = ex * ex + ey * ey + ez * ez <= rbox2;
                }
                const unsigned bal = __ballot_sync(full, keep);
                if (keep) {
                    const int pos = ncand + __popc(bal & lt_mask);
                    cl[pos] = rec;
                    ch[pos] = sh;
                    cll[pos] = shl;
                    cp[pos] = make_float4((float)rec.xh, (float)rec.yh, (float)rec.zh + shf, (float)rec.q);
                }
                ncand += __popc(bal);
                if (ncand >= 64) {
                    process(ncand);
                    ncand = 0;
                }
            }
        }
    }
    if (ncand > 0) process(ncand);
    if (valid) {
        // the kRealSplit warps of a target group combine through FP64 atomics
        // (outputs are zeroed beforehand when not accumulating)
        const double qm = (accumulate & 2) ? 1.0 : (double)me.q;  // bit 1: field instead of force
        const int o = me.orig;
        atomicAdd(phi + o, aphi);
        atomicAdd(frc + 3 * o, qm * afx);
        atomicAdd(frc + 3 * o + 1, qm * afy);
        atomicAdd(frc + 3 * o + 2, qm * afz);
    }
    (void)accumulate;
}

}  // namespace

template <typename T>
void launch_real_space(se1p_plan *p, int n, const int *cell_key, double *phi, double *frc, int accumulate,
                       cudaStream_t s)
{
    const Geo &g = p->geo;
    if (n <= 0) return;
    if (!(accumulate & 1)) {
        cudaMemsetAsync(phi, 0, sizeof(double) * (size_t)n, s);
        cudaMemsetAsync(frc, 0, sizeof(double) * 3 * (size_t)n, s);
    }
    const int warps = (n + 31) / 32 * kRealSplit;
    k_real<T><<<(warps + kRealWarps - 1) / kRealWarps, 32 * kRealWarps, 0, s>>>(
        g, n, p->b.starts + g.nbins + 1, (const CellRec<T> *)p->b.cells, cell_key, phi, frc, accumulate);
}

template void launch_real_space<float>(se1p_plan *, int, const int *, double *, double *, int, cudaStream_t);
template void launch_real_space<double>(se1p_plan *, int, const int *, double *, double *, int, cudaStream_t);

}  // namespace se1p
