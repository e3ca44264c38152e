// Real-space part of the Ewald1P sum (Eq. 2.2) and its force (Eq. 3.22) over
// a cell list (Section 3: linked cells no smaller than rc, z images by
// unwrapped neighbour-cell indices).
#include <cuda_runtime.h>
#include <math.h>

#include "se1p_plan.h"

namespace se1p {

namespace {

constexpr int kRealWarps = 4;  // warps per CTA (warps work independently)
// Warps sharing one group of targets (SPLIT, a template parameter: the source rows are split
// between them and FP64 atomics combine their sums).  Four pay where a target has many neighbours,
// two where the grid path dominates; measured beside the grid path: N = 10^5 in the unit box,
// rc = 0.15 (~1400 expected neighbours): 1.528 ms with four, 1.543 with two; N = 10^6 in [1,1,8],
// rc = 0.09 (~380): 12.42 ms with four, 12.32 with two.
constexpr double kRealSplitNeighbours = 800.0;
// One warp per target group below this (64 systems of ~230 expected neighbours: 14.86 -> 14.78 ms;
// N = 10^6 in [1, 1, 8] with ~380 keeps two: 10.57 against 10.60 ms with one)
constexpr double kRealOneWarpNeighbours = 300.0;
// CTAs per SM the FP32 kernel is compiled for (72 registers per thread): with the unrolled candidate
// test the compiler would take 96 and fit five; seven are faster (C2, stage alone: 0.83 against 0.96 ms)
constexpr int kCand = 96;      // per-warp candidate list (flushed at >= 64)
constexpr int kRealTargets = 16;                     // targets per warp
constexpr int kLanesPerTarget = 32 / kRealTargets;   // lanes sharing a target (alternate candidates)

// Hardware approximations with denormals flushed (arguments here are far from the
// denormal range: r^2 >= ~1e-14, exp(-xi^2 r^2) >= ~1e-11, 1 + x/2 >= 1).
__device__ __forceinline__ float rsqrt_hw(float v)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}
__device__ __forceinline__ float ex2_hw(float v)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}
__device__ __forceinline__ float rcp_hw(float v)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(v));
    return y;
}

template <typename T> __device__ __forceinline__ T exp_t(T v);
template <> __device__ __forceinline__ float exp_t<float>(float v) { return ex2_hw(v * 1.4426950408889634f); }
template <> __device__ __forceinline__ double exp_t<double>(double v) { return exp(v); }

template <typename T> __device__ __forceinline__ T rsqrt_t(T v);
// 1/sqrt with one Newton step after the hardware estimate, so that r = r2 / sqrt(r2)
// is within ~1 ulp (erfc(xi r) near rc amplifies the relative error of r ~10x).
template <> __device__ __forceinline__ float rsqrt_t<float>(float v)
{
    const float y = rsqrt_hw(v);
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
    float t = rcp_hw(d);
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

// A source (with its z image shift folded in) or a target, in shared memory:
// hi parts and the charge first, so the hi float4 doubles as the phase-1 copy.
template <typename T> struct __align__(sizeof(T) == 4 ? 16 : 32) PairRec {
    T xh, yh, zh, q;
    T xl, yl, zl, pad;
};

// Displacement target - source from hi + lo parts.  Each hi difference is one
// rounding of a difference (exact when the two are within a factor 2, Sterbenz),
// the lo parts restore the FP64 coordinates to ~1e-15.  In FP64 the lo parts hold
// only the rounding errors of image shifts: z always, x and y for triply periodic plans.
template <typename T>
__device__ __forceinline__ void displacement(const PairRec<T> &a, const PairRec<T> &c, T &dx, T &dy, T &dz, bool per3)
{
    dx = a.xh - c.xh;
    dy = a.yh - c.yh;
    dz = a.zh - c.zh;
    if (sizeof(T) < sizeof(double) || per3) {
        dx += a.xl - c.xl;
        dy += a.yl - c.yl;
    }
    dz += a.zl - c.zl;
}

// v + shift as hi + lo: Fast2Sum (|sh| >= |v| whenever sh != 0, since v lies in [0, L) and sh is a
// whole number of periods) gives the rounding error of the hi sum exactly
template <typename T> __device__ __forceinline__ void shifted(T vh, T vl, T sh, T shl, T &oh, T &ol)
{
    oh = sh + vh;
    ol = (vl + shl) + (vh - (oh - sh));
}

__device__ __forceinline__ int floor_div(int a, int m) { return a >= 0 ? a / m : -((-a + m - 1) / m); }

// Contribution of one source of charge qs at displacement d (Eq. 2.2 and its
// gradient, Eq. 3.22), added to (ph, fx, fy, fz).  Pairs with r = 0 (the target
// itself; distinct coincident charges are outside the sum's domain) or r > rc
// add nothing.  Branch-free: rejected pairs run on r^2 = rc^2 with zero charge.
template <typename T>
__device__ __forceinline__ void pair_terms(T dx, T dy, T dz, T qs, T rc2, T xi, T xi2, T two_xi_sqpi, T &ph,
                                           T &fx, T &fy, T &fz)
{
    const T r2 = dx * dx + dy * dy + dz * dz;
    const bool ok = r2 > (T)0 && r2 <= rc2;
    const T r2s = ok ? r2 : rc2;
    const T qq = ok ? qs : (T)0;
    const T rinv = rsqrt_t<T>(r2s);
    const T r = r2s * rinv;
    const T E = exp_t<T>(-xi2 * r2s);
    const T e = erfc_from_exp(xi * r, E) * rinv;
    ph += qq * e;
    const T fs = qq * (two_xi_sqpi * E + e) * rinv * rinv;
    fx += fs * dx;
    fy += fs * dy;
    fz += fs * dz;
}

// Pair terms without charges, for the evaluation of each pair once: e = erfc(xi r) / r and
// g = (2 xi / sqrt(pi) exp(-xi^2 r^2) + e) / r^2, so that a source of charge q adds q e to the
// target's potential and q g d to its field, and the target adds q_t e and -q_t g d to the source's;
// e = g = 0 where r = 0 or r > rc.
template <typename T>
__device__ __forceinline__ void pair_terms_eg(T dx, T dy, T dz, T rc2, T xi, T xi2, T two_xi_sqpi, T &e, T &g)
{
    const T r2 = dx * dx + dy * dy + dz * dz;
    const bool ok = r2 > (T)0 && r2 <= rc2;
    const T r2s = ok ? r2 : rc2;
    const T rinv = rsqrt_t<T>(r2s);
    const T r = r2s * rinv;
    const T E = exp_t<T>(-xi2 * r2s);
    const T ev = erfc_from_exp(xi * r, E) * rinv;
    e = ok ? ev : (T)0;
    g = ok ? (two_xi_sqpi * E + ev) * rinv * rinv : (T)0;
}

// Source-side sums of one listed candidate (FP64): phi, then the field (x, y, z), added to by the
// lanes of the warp concurrently.
struct __align__(32) SrcAcc {
    double v[4];
};
__device__ __forceinline__ void slot_add(SrcAcc *s, double a, double b, double c, double d)
{
    atomicAdd(&s->v[0], a);
    atomicAdd(&s->v[1], b);
    atomicAdd(&s->v[2], c);
    atomicAdd(&s->v[3], d);
}

// Real-space sum, warp-centric.  Warp w owns the kRealTargets consecutive targets
// from kRealTargets w in cell order (any cell boundaries), so its targets occupy a
// small box of cells; kLanesPerTarget lanes share a target and take alternate
// candidates.  Sources come from that box expanded by
// S = ceil(rc / cell edge) cells per axis; for each (y, z) cell row the x-range
// is contiguous in cell order, i.e. one source range; z images come from
// unwrapped rows nz_u = nz + wrap * ncz, shifted by wrap * L3 (folded into the
// source's z as an exact hi + lo sum, Fast2Sum).
//
// Sources are read 32 at a time, one per lane, and tested in parallel against
// the warp's target bounding box grown by rc; the survivors are compacted by
// ballot into a per-warp list.  When the list holds >= 64 candidates:
//   phase 1: every lane marks its share of the candidates within rc of its target
//            (float test on the hi parts, threshold widened so no true pair is lost);
//   phase 2: every lane walks its own marks: hi + lo displacement, the exact
//            r <= rc test and the pair terms, branch-free.
// (Spreading the marks of busy lanes over idle ones through shared memory was
// measured slower: the bookkeeping per pair costs more than the idle lanes.)
//
// FP64 (SYM) evaluates each pair once, from the end that finds it: the potential term of a pair is
// the same for both particles and the force term opposite.  Pair rule: source j at image shift s
// pairs with target i in this warp when key(j, s) > 2 i, with key(j, s) = 2 j + [s > 0] (shifts
// ordered lexicographically by their z, y, x images).  Of a pair (i, j, s) and its mirror
// (j, i, -s) exactly one passes, and of a particle's own images (j = i) those with s > 0, each
// counted for both ends.  So every source range starts at the warp's first target, and only
// candidates that are the warp's own targets need the key test.  Phase 2 adds the source's terms
// to the candidate's slot in shared memory (atomic adds; the lanes walk their marks from
// different starting bits, so that nearby targets, which mark the same candidates, do not queue
// on one slot); after the walk the slots go to the sums in cell order, rsum (FP64 atomics on
// consecutive indices, mostly), which k_real_out maps to the caller's order.  Halves the FP64
// real space (N = 10^5, alone: 22.7 against 38.6 ms).  FP32 keeps evaluating each pair from both
// ends: its source-side sums would need shared-memory atomics (0.98 against 0.84 ms), a per-warp
// matrix of terms (32 KB per CTA, which keeps the gridding kernels off the SMs beside it: the
// overlapped evaluation took 1.72 against 1.46 ms), or a second walk over the transposed marks
// (0.77 ms alone, but 1.52 against 1.48 ms for the overlapped evaluation and 3.60 against 3.43 ms
// alone at N = 10^6 in [1, 1, 8]).
constexpr int kRealMinBlocks32 = 7;

template <typename T, int SPLIT, bool PER3>
__global__ void __launch_bounds__(32 * kRealWarps, sizeof(T) == 4 ? kRealMinBlocks32 : 1) k_real(Geo g, int n, const int *__restrict__ cell_start,
                                                          const CellRec<T> *__restrict__ cells,
                                                          const int *__restrict__ cell_key,
                                                          double *__restrict__ phi, double *__restrict__ frc,
                                                          int accumulate, double *__restrict__ rsum)
{
    constexpr bool SYM = sizeof(T) == sizeof(double);  // each pair once
    __shared__ PairRec<T> cand[kRealWarps][kCand];
    __shared__ int ckey[SYM ? kRealWarps : 1][SYM ? kCand : 1];  // key(j, s) of the listed candidates
    __shared__ SrcAcc sacc[SYM ? kRealWarps : 1][SYM ? 64 : 1];  // source-side sums of a flush
    __shared__ float4 cposd[sizeof(T) == 4 ? 1 : kRealWarps][sizeof(T) == 4 ? 1 : kCand];  // FP64: float copy
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * kRealWarps + wib;
    const int warp = gw / SPLIT, part = gw % SPLIT;  // target group, share of the source rows
    const int half = lane / kRealTargets;  // which share of the candidates this lane takes
    const int t = warp * kRealTargets + lane % kRealTargets;
    if (warp * kRealTargets >= n) return;  // whole warp beyond the particles
    const bool valid = t < n;
    const int a0 = warp * kRealTargets;  // first target of the group
    int *key = ckey[SYM ? wib : 0];
    SrcAcc *acc = sacc[SYM ? wib : 0];
    if constexpr (SYM)
        for (int j = lane; j < 64; j += 32) acc[j] = SrcAcc{{0.0, 0.0, 0.0, 0.0}};
    const int mykey = 2 * t;
    const int own_end = 2 * (a0 + kRealTargets);  // keys below: the warp's own targets
    PairRec<T> me;
    int orig = -1;
    T qme = (T)0;
    int cx = 0, cy = 0, cz = 0;
    if (valid) {
        const CellRec<T> r = cells[t];
        me.xh = r.xh;
        me.yh = r.yh;
        me.zh = r.zh;
        me.xl = r.xl;
        me.yl = r.yl;
        me.zl = r.zl;
        qme = r.q;
        orig = r.orig;
        const int cell = cell_key[orig];
        cx = cell % g.ncx;
        cy = (cell / g.ncx) % g.ncy;
        cz = cell / (g.ncx * g.ncy);
    } else {
        me.xh = me.yh = me.zh = me.xl = me.yl = me.zl = (T)0;
    }
    me.q = me.pad = (T)0;
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
    // unwrapped cell ranges: clamped to the box on the free axes (SE1P), periodic images on every
    // axis of a triply periodic plan; an x range that crosses the box edge splits into segments
    constexpr bool per3 = PER3;  // triply periodic plan (g.per3)
    const int nx_lo = per3 ? cx0 - Sx : max(cx0 - Sx, 0), nx_hi = per3 ? cx1 + Sx : min(cx1 + Sx, g.ncx - 1);
    const int ny_lo = per3 ? cy0 - Sy : max(cy0 - Sy, 0), ny_hi = per3 ? cy1 + Sy : min(cy1 + Sy, g.ncy - 1);
    const int wx0 = per3 ? floor_div(nx_lo, g.ncx) : 0, nseg = per3 ? floor_div(nx_hi, g.ncx) - wx0 + 1 : 1;
    const T xi = (T)g.xi, rc2 = (T)g.rc2;
    const T two_xi_sqpi = (T)(2.0 * g.xi / sqrt(kPi));
    const T xi2 = (T)(g.xi * g.xi);
    PairRec<T> *cl = cand[wib];
    const float4 *cp = sizeof(T) == 4 ? reinterpret_cast<const float4 *>(cl) : cposd[sizeof(T) == 4 ? 0 : wib];
    constexpr int cps = sizeof(T) == 4 ? 2 : 1;  // float4 stride of the phase-1 copy
    const unsigned lt_mask = (1u << lane) - 1u;
    double aphi = 0, afx = 0, afy = 0, afz = 0;
    int ncand = 0;

    const float mxf = (float)me.xh, myf = (float)me.yh, mzf = (float)me.zh;
    // phase-1 threshold: rc widened by 1e-5 rc plus a few float ulps of the box size, so the
    // float test (coordinates and image shift rounded to float) never drops a true pair
    const double lmax = fmax(fmax(g.L[0], g.L[1]), g.L[2]);
    const float rc2wf = (float)((g.rc * (1.0 + 1e-5) + 5e-7 * lmax) * (g.rc * (1.0 + 1e-5) + 5e-7 * lmax));

    auto process = [&](int nc) {  // nc <= 64 candidates in cl[0 .. nc)
        __syncwarp();
        // phase 1: candidates within rc of this lane's target (float test, widened threshold); this
        // lane's candidate k kLanesPerTarget + half is bit k of its marks.  Always 64 / kLanesPerTarget
        // tests, unrolled, then the bits beyond nc are cleared (the list past nc holds stale records).
        unsigned m0 = 0u;
        if (valid) {
#pragma unroll
            for (int k = 0; k < 64 / kLanesPerTarget; ++k) {
                const float4 c = cp[(k * kLanesPerTarget + half) * cps];
                const float dx = mxf - c.x, dy = myf - c.y, dz = mzf - c.z;
                if (dx * dx + dy * dy + dz * dz <= rc2wf) m0 |= 1u << k;
            }
            const int nk = (nc - half + kLanesPerTarget - 1) / kLanesPerTarget;
            if (nk < 32) m0 &= (1u << max(nk, 0)) - 1u;
        }
        int rot = 0;
        if constexpr (SYM) {
            // the pair rule, needed only where the list holds the warp's own targets
            const bool own = (lane < nc && key[lane] < own_end) || (lane + 32 < nc && key[lane + 32] < own_end);
            if (__any_sync(full, own)) {
                unsigned mm = m0;
                while (mm) {
                    const int k = __ffs(mm) - 1;
                    mm &= mm - 1u;
                    if (key[k * kLanesPerTarget + half] <= mykey) m0 &= ~(1u << k);
                }
            }
            rot = lane % kRealTargets;  // the walk starts at bit rot, cyclically
            m0 = __funnelshift_r(m0, m0, rot);
        }
        // phase 2: this lane's marks, word by word
        T pphi = 0, pfx = 0, pfy = 0, pfz = 0;
        auto walk = [&](unsigned m, int k0) {
            while (m) {
                const int j = (SYM ? ((k0 + __ffs(m) - 1 + rot) & 31) : k0 + __ffs(m) - 1) * kLanesPerTarget + half;
                m &= m - 1u;
                T dx, dy, dz;
                displacement(me, cl[j], dx, dy, dz, per3);
                if constexpr (SYM) {
                    T e, gq;
                    pair_terms_eg(dx, dy, dz, rc2, xi, xi2, two_xi_sqpi, e, gq);
                    const T qs = cl[j].q;
                    pphi += qs * e;
                    const T gs = qs * gq;
                    pfx += gs * dx;
                    pfy += gs * dy;
                    pfz += gs * dz;
                    const T gt = qme * gq;
                    slot_add(acc + j, qme * e, -(gt * dx), -(gt * dy), -(gt * dz));
                } else {
                    pair_terms(dx, dy, dz, cl[j].q, rc2, xi, xi2, two_xi_sqpi, pphi, pfx, pfy, pfz);
                }
            }
        };
        walk(m0, 0);
        aphi += (double)pphi;
        afx += (double)pfx;
        afy += (double)pfy;
        afz += (double)pfz;
        __syncwarp();
        if constexpr (SYM) {
            // the nc candidates' source-side sums into the sums in cell order; the slots start over
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j < nc) {
                    const SrcAcc v = acc[j];
                    acc[j] = SrcAcc{{0.0, 0.0, 0.0, 0.0}};
                    const int si = key[j] >> 1;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (v.v[c] != 0.0) atomicAdd(rsum + (size_t)c * n + si, v.v[c]);
                }
            }
            __syncwarp();
        }
    };

    const int nyr = ny_hi - ny_lo + 1;
    const int nrows = (cz1 + Sz - (cz0 - Sz) + 1) * max(nyr, 0) * nseg;
    for (int rr = part; rr < nrows; rr += SPLIT) {
        const int seg = rr % nseg, ryz = rr / nseg;
        const int nzu = cz0 - Sz + ryz / nyr, nyu = ny_lo + ryz % nyr;
        const int wrap = floor_div(nzu, g.ncz), wy = per3 ? floor_div(nyu, g.ncy) : 0, wx = wx0 + seg;
        const int nz = nzu - wrap * g.ncz, ny = nyu - wy * g.ncy;
        // image shift s > 0 (lexicographic in z, y, x): the key's low bit
        const int spos = (wrap > 0 || (wrap == 0 && (wy > 0 || (wy == 0 && wx > 0)))) ? 1 : 0;
        const double shd = wrap * g.L[2];
        const T sh = (T)shd, shl = (T)(shd - (double)sh);
        const float shf = (float)shd;
        // x and y image shifts (zero for SE1P)
        const double sxd = per3 ? wx * g.L[0] : 0.0, syd = per3 ? wy * g.L[1] : 0.0;
        const T sxh = (T)sxd, sxl = (T)(sxd - (double)sxh), syh = (T)syd, syl = (T)(syd - (double)syh);
        const float sxf = (float)sxd, syf = (float)syd;
        const int xa = per3 ? max(nx_lo, wx * g.ncx) - wx * g.ncx : nx_lo;
        const int xb = per3 ? min(nx_hi, wx * g.ncx + g.ncx - 1) - wx * g.ncx : nx_hi;
        const int row = (nz * g.ncy + ny) * g.ncx;
        // SYM: sources before the warp's first target pair with it in their own warps
        const int sbeg = SYM ? max(cell_start[row + xa], a0) : cell_start[row + xa], send = cell_start[row + xb + 1];
        for (int s0 = sbeg; s0 < send; s0 += 32) {
            bool keep = false;
            const int si = s0 + lane;
            const bool have = si < send;
            CellRec<T> rec;
            if (have) rec = cells[si];
            float sx = 0.f, sy = 0.f, sz = 0.f;
            if (have) {
                sx = (float)rec.xh + sxf;
                sy = (float)rec.yh + syf;
                sz = (float)rec.zh + shf;
                const float ex = fmaxf(fmaxf(bx0 - sx, sx - bx1), 0.0f);
                const float ey = fmaxf(fmaxf(by0 - sy, sy - by1), 0.0f);
                const float ez = fmaxf(fmaxf(bz0 - sz, sz - bz1), 0.0f);
                keep = ex * ex + ey * ey + ez * ez <= rbox2;
            }
            const unsigned bal = __ballot_sync(full, keep);
            if (keep) {
                const int pos = ncand + __popc(bal & lt_mask);
                PairRec<T> c;
                shifted(rec.zh, rec.zl, sh, shl, c.zh, c.zl);
                if constexpr (per3) {
                    shifted(rec.xh, rec.xl, sxh, sxl, c.xh, c.xl);
                    shifted(rec.yh, rec.yl, syh, syl, c.yh, c.yl);
                } else {
                    c.xh = rec.xh;
                    c.xl = rec.xl;
                    c.yh = rec.yh;
                    c.yl = rec.yl;
                }
                c.q = rec.q;
                c.pad = (T)0;
                cl[pos] = c;
                if constexpr (SYM) key[pos] = 2 * si + spos;
                if constexpr (sizeof(T) != 4)
                    cposd[sizeof(T) == 4 ? 0 : wib][sizeof(T) == 4 ? 0 : pos] = make_float4(sx, sy, sz, (float)rec.q);
            }
            ncand += __popc(bal);
            if (ncand >= 64) {
                process(64);
                // the candidates beyond the first 64 (fewer than 32) move to the front of the list
                const int rest = ncand - 64;
                PairRec<T> tmp;
                float4 tmpd;
                int tk = 0;
                if (lane < rest) {
                    tmp = cl[64 + lane];
                    if constexpr (SYM) tk = key[64 + lane];
                    if constexpr (sizeof(T) != 4) tmpd = cposd[sizeof(T) == 4 ? 0 : wib][sizeof(T) == 4 ? 0 : 64 + lane];
                }
                __syncwarp();
                if (lane < rest) {
                    cl[lane] = tmp;
                    if constexpr (SYM) key[lane] = tk;
                    if constexpr (sizeof(T) != 4) cposd[sizeof(T) == 4 ? 0 : wib][sizeof(T) == 4 ? 0 : lane] = tmpd;
                }
                __syncwarp();
                ncand = rest;
            }
        }
    }
    if (ncand > 0) process(ncand);
#pragma unroll
    for (int o = kRealTargets; o < 32; o <<= 1) {  // lanes sharing a target
        aphi += __shfl_xor_sync(full, aphi, o);
        afx += __shfl_xor_sync(full, afx, o);
        afy += __shfl_xor_sync(full, afy, o);
        afz += __shfl_xor_sync(full, afz, o);
    }
    if (valid && half == 0) {
        if constexpr (SYM) {
            // the SPLIT warps of a target group and the warps holding this target as a source all
            // add into the sums in cell order (zeroed before the launch)
            atomicAdd(rsum + t, aphi);
            atomicAdd(rsum + (size_t)n + t, afx);
            atomicAdd(rsum + 2 * (size_t)n + t, afy);
            atomicAdd(rsum + 3 * (size_t)n + t, afz);
        } else {
            // the SPLIT warps of a target group combine through FP64 atomics
            // (outputs are zeroed beforehand when not accumulating)
            const double qm = (accumulate & 2) ? 1.0 : (double)qme;  // bit 1: field instead of force
            atomicAdd(phi + orig, aphi);
            atomicAdd(frc + 3 * orig, qm * afx);
            atomicAdd(frc + 3 * orig + 1, qm * afy);
            atomicAdd(frc + 3 * orig + 2, qm * afz);
        }
    }
}

// FP64 sums in cell order -> caller order: phi, and q times the field (the force) or the field
// itself (flags bit 1); overwritten, or added (flags bit 0).
__global__ void k_real_out(int n, const CellRec<double> *__restrict__ cells, const double *__restrict__ rsum,
                           double *__restrict__ phi, double *__restrict__ frc, int flags)
{
    const int si = blockIdx.x * blockDim.x + threadIdx.x;
    if (si >= n) return;
    const int o = cells[si].orig;
    const double qm = (flags & 2) ? 1.0 : cells[si].q;
    const double ph = rsum[si], fx = qm * rsum[(size_t)n + si], fy = qm * rsum[2 * (size_t)n + si],
                 fz = qm * rsum[3 * (size_t)n + si];
    if (flags & 1) {
        phi[o] += ph;
        frc[3 * (size_t)o] += fx;
        frc[3 * (size_t)o + 1] += fy;
        frc[3 * (size_t)o + 2] += fz;
    } else {
        phi[o] = ph;
        frc[3 * (size_t)o] = fx;
        frc[3 * (size_t)o + 1] = fy;
        frc[3 * (size_t)o + 2] = fz;
    }
}

}  // namespace

template <typename T>
void launch_real_space(se1p_plan *p, int n, const int *cell_key, double *phi, double *frc, int accumulate,
                       cudaStream_t s)
{
    const Geo &g = p->geo;
    if (n <= 0) return;
    constexpr bool sym = sizeof(T) == sizeof(double);  // each pair once, sums in cell order
    double *rsum = p->b.rsum;
    if (sym) {
        cudaMemsetAsync(rsum, 0, sizeof(double) * 4 * (size_t)n, s);
    } else if (!(accumulate & 1)) {
        cudaMemsetAsync(phi, 0, sizeof(double) * (size_t)n, s);
        cudaMemsetAsync(frc, 0, sizeof(double) * 3 * (size_t)n, s);
    }
    // expected neighbours of a target within rc at uniform density
    const double neighbours = n / (g.L[0] * g.L[1] * g.L[2]) * 4.0 / 3.0 * kPi * g.rc * g.rc * g.rc;
    const int groups = (n + kRealTargets - 1) / kRealTargets;
    const int *starts = p->b.starts + g.nbins + 1;
    const CellRec<T> *cells = (const CellRec<T> *)p->b.cells;
    if (neighbours >= kRealSplitNeighbours) {
        const int blocks = (groups * 4 + kRealWarps - 1) / kRealWarps;
        if (g.per3) k_real<T, 4, true><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
        else k_real<T, 4, false><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
    } else if (neighbours < kRealOneWarpNeighbours) {
        const int blocks = (groups + kRealWarps - 1) / kRealWarps;
        if (g.per3) k_real<T, 1, true><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
        else k_real<T, 1, false><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
    } else {
        const int blocks = (groups * 2 + kRealWarps - 1) / kRealWarps;
        if (g.per3) k_real<T, 2, true><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
        else k_real<T, 2, false><<<blocks, 32 * kRealWarps, 0, s>>>(g, n, starts, cells, cell_key, phi, frc, accumulate, rsum);
    }
    if constexpr (sym)
        k_real_out<<<(n + 255) / 256, 256, 0, s>>>(n, reinterpret_cast<const CellRec<double> *>(cells), rsum, phi, frc,
                                                   accumulate);
}

template void launch_real_space<float>(se1p_plan *, int, const int *, double *, double *, int, cudaStream_t);
template void launch_real_space<double>(se1p_plan *, int, const int *, double *, double *, int, cudaStream_t);

}  // namespace se1p
