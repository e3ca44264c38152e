// C ABI of libse1p: plan creation (parameter resolution of Section 4.3,
// workspace, FP64 k3 = 0 table), orchestration of Algorithm 1 plus the real
// space and self terms, and the single-step entry points.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "se1p_plan.h"

using namespace se1p;

namespace {

constexpr double kShapeC = 0.95;  // Gaussian shape constant c of Eq. 3.3
// shared memory per Fourier-pass CTA: small enough that the passes find room on SMs that the
// concurrent real space occupies (measured at N = 10^6, M3 = 1024: 32 / 48 / 64 / 96 KB 10.59 / 10.56 /
// 10.45 / 10.60 ms; 64 systems 15.24 / 14.73 / 14.72 / 15.42 ms; N = 10^5 unchanged)
constexpr size_t kSmemBudget = 64 * 1024;

bool is_smooth(long n)
{
    if (n < 1) return false;
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) n /= p;
    return n == 1;
}

int next_smooth(long n)
{
    if (n < 1) n = 1;
    while (!is_smooth(n)) ++n;
    return (int)n;
}

bool make_fft(int n, FftDesc &d)
{
    if (!is_smooth(n)) return false;
    d.n = n;
    d.nrad = 0;
    int m = n;
    auto push = [&](int r) {
        if (d.nrad >= 24) return false;
        d.rad[d.nrad++] = r;
        return true;
    };
    while (m % 8 == 0) { if (!push(8)) return false; m /= 8; }
    while (m % 4 == 0) { if (!push(4)) return false; m /= 4; }
    while (m % 2 == 0) { if (!push(2)) return false; m /= 2; }
    for (int r : {3, 5, 7})
        while (m % r == 0) { if (!push(r)) return false; m /= r; }
    if (m != 1) return false;
    int Ns = 1;
    for (int st = 0; st < d.nrad; ++st) {
        d.ns[st] = make_fastdiv((unsigned)Ns);
        d.nb[st] = make_fastdiv((unsigned)(n / d.rad[st]));
        Ns *= d.rad[st];
    }
    return true;
}

template <typename T> size_t csize() { return sizeof(Cx<T>); }

int pow2_fit(size_t per_unit, int cap)
{
    int v = cap;
    while (v > 1 && per_unit * v > kSmemBudget) v >>= 1;
    return v;
}

// Workspace allocator of plan creation.  Every allocation is recorded in the plan, so a failure
// part-way frees everything allocated before it.  For tests of that path, the environment variable
// SE1P_TEST_FAIL_ALLOC = k (k >= 1) makes the k-th allocation of each plan creation fail as if the
// device or host were out of memory (nothing is requested from CUDA for it).
struct Alloc {
    se1p_plan *p;
    bool ok = true;
    int count = 0, fail_at = 0;
    bool injected()
    {
        if (++count == fail_at) {
            ok = false;
            return true;
        }
        return false;
    }
    void *dev(size_t bytes)
    {
        if (!ok || bytes == 0) return nullptr;
        if (injected()) return nullptr;
        void *ptr = nullptr;
        if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        p->dev_allocs.push_back(ptr);
        p->bytes += bytes;
        return ptr;
    }
    void *pinned(size_t bytes)  // page-locked host memory
    {
        if (!ok || bytes == 0) return nullptr;
        if (injected()) return nullptr;
        void *ptr = nullptr;
        if (cudaMallocHost(&ptr, bytes) != cudaSuccess) {
            ok = false;
            cudaGetLastError();
            return nullptr;
        }
        p->host_allocs.push_back(ptr);
        return ptr;
    }
};

void free_all(se1p_plan *p)
{
    for (void *ptr : p->dev_allocs) cudaFree(ptr);
    p->dev_allocs.clear();
    for (void *ptr : p->host_allocs) cudaFreeHost(ptr);
    p->host_allocs.clear();
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->s_real) cudaStreamDestroy(p->s_real);
    p->ev_fork = p->ev_join = nullptr;
    p->s_real = nullptr;
    for (int i = 0; i < 3; ++i) {
        if (p->ev_f[i]) cudaEventDestroy(p->ev_f[i]);
        p->ev_f[i] = nullptr;
    }
    for (int i = 0; i < 2; ++i) {
        if (p->s_f[i]) cudaStreamDestroy(p->s_f[i]);
        p->s_f[i] = nullptr;
    }
}

template <typename T> void upload(void *dst, const std::vector<T> &v)
{
    cudaMemcpy(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

template <typename T> std::vector<Tw<T>> twiddles(int n)
{
    std::vector<Tw<T>> w(n);
    for (int t = 0; t < n; ++t) {
        const double a = 2.0 * kPi * (double)t / (double)n;
        const double c = cos(a), sn = -sin(a);
        w[t].re = (T)c;
        w[t].im = (T)sn;
        if constexpr (sizeof(T) == sizeof(float)) {
            w[t].lre = (float)(c - (double)w[t].re);
            w[t].lim = (float)(sn - (double)w[t].im);
        }
    }
    return w;
}

template <typename T> se1p_status build_tables(se1p_plan *p, Alloc &A)
{
    // twiddles
    p->b.tw_z = A.dev(sizeof(Tw<T>) * p->M3);
    for (int c = 0; c < 3; ++c) {
        SlabClass &C = p->cls[c];
        if (C.count == 0) continue;
        C.tw = A.dev((c == 0 ? sizeof(Tw<double>) : sizeof(Tw<T>)) * C.ns);
        C.rows = A.dev((c == 0 ? csize<double>() : csize<T>()) * (size_t)C.count * p->Mf * C.ns);
        if (c > 0) C.sym = A.dev(sizeof(T) * (size_t)C.count * C.ns * C.ns);
    }
    if (!A.ok) return SE1P_ERR_ALLOC;
    upload(p->b.tw_z, twiddles<T>(p->M3));
    for (int c = 0; c < 3; ++c) {
        SlabClass &C = p->cls[c];
        if (C.count == 0) continue;
        if (c == 0) upload(C.tw, twiddles<double>(C.ns));
        else upload(C.tw, twiddles<T>(C.ns));
    }
    return SE1P_OK;
}

template <typename T> se1p_status alloc_particles(se1p_plan *p, Alloc &A)
{
    const int nm = p->n_max > 0 ? p->n_max : 1;
    const Geo &g = p->geo;
    p->b.grid = A.dev(sizeof(T) * grid_points(p->M3, p->Mt));
    p->b.gridf = p->per3 ? A.dev(sizeof(T) * grid_points(p->M3, p->Mf)) : p->b.grid;
    p->b.zspec = A.dev(csize<T>() * (size_t)p->K3 * p->Mf * p->Mf);
    p->b.slab0_in = (double *)A.dev(sizeof(double) * (size_t)p->Mf * p->Mf);
    p->b.slab0_out = (double *)A.dev(sizeof(double) * (size_t)p->Mf * p->Mf);
    p->b.sym0 = (double *)A.dev(sizeof(double) * (size_t)p->n0 * p->n0);
    p->b.xyzq = (double *)A.dev(sizeof(double) * 4 * (size_t)nm);
    p->b.bin_key = (int *)A.dev(sizeof(int) * (size_t)nm);
    p->b.cell_key = (int *)A.dev(sizeof(int) * (size_t)nm);
    p->b.counts = (int *)A.dev(sizeof(int) * (size_t)(g.nbins + g.ncells));
    p->b.starts = (int *)A.dev(sizeof(int) * (size_t)(g.nbins + g.ncells + 2));
    p->b.cursors = (int *)A.dev(sizeof(int) * (size_t)(g.nbins + g.ncells));
    p->b.scan_tmp = (int *)A.dev(sizeof(int) * (size_t)kScanTmp);
    p->b.gchunk = (int *)A.dev(sizeof(int) * (size_t)kGatherChunks);
    p->b.parts = A.dev(sizeof(PartRec<T>) * (size_t)nm);
    p->b.wts = A.dev(sizeof(T) * 3 * (size_t)p->geo.P * nm);
    p->b.cells = A.dev(sizeof(CellRec<T>) * (size_t)nm);
    p->b.phi_int = (double *)A.dev(sizeof(double) * (size_t)nm);
    p->b.frc_int = (double *)A.dev(sizeof(double) * 3 * (size_t)nm);
    p->b.phi2 = (double *)A.dev(sizeof(double) * (size_t)nm);
    p->b.frc2 = (double *)A.dev(sizeof(double) * 3 * (size_t)nm);
    if (sizeof(T) == sizeof(double)) p->b.rsum = (double *)A.dev(sizeof(double) * 4 * (size_t)nm);
    p->b.sums = (double *)A.dev(sizeof(double) * 2);
    p->b.epart = (double *)A.dev(sizeof(double) * kEnergyBlocks);
    p->b.status = (int *)A.dev(sizeof(int));
    p->b.hstatus = (int *)A.pinned(sizeof(int));
    p->b.hx = (double *)A.dev(sizeof(double) * 3 * (size_t)nm);
    p->b.hq = (double *)A.dev(sizeof(double) * (size_t)nm);
    p->b.hphi = (double *)A.dev(sizeof(double) * (size_t)nm);
    p->b.hfrc = (double *)A.dev(sizeof(double) * 3 * (size_t)nm);
    p->b.hen = (double *)A.dev(sizeof(double));
    if (!A.ok) return SE1P_ERR_ALLOC;
    cudaMemset(p->b.status, 0, sizeof(int));
    // the x padding of the last block of each grid row stays zero (kernels write only x < Mt)
    cudaMemset(p->b.grid, 0, sizeof(T) * grid_points(p->M3, p->Mt));
    if (p->per3) cudaMemset(p->b.gridf, 0, sizeof(T) * grid_points(p->M3, p->Mf));
    return SE1P_OK;
}

se1p_status check_launch()
{
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SE1P_OK : SE1P_ERR_CUDA;
}

// ---------------------------------------------------------------- orchestration
constexpr int kProfMaxEvals = 4096;
constexpr int kProfEventsPerEval = 2 * SE1P_NUM_STAGES;

// Start and end events of each stage of one evaluation, recorded on the stream the stage runs on
// (the real space overlaps the grid path, so stage times may add up to more than the evaluation).
struct StageMarks {
    se1p_plan *p;
    bool on;
    explicit StageMarks(se1p_plan *p_) : p(p_), on(p_->profiling && p_->prof_count < kProfMaxEvals) {}
    void begin(int stage, cudaStream_t s) { record(2 * stage, s); }
    void end(int stage, cudaStream_t s) { record(2 * stage + 1, s); }
    void record(int k, cudaStream_t s)
    {
        if (on) cudaEventRecord(p->prof_events[(size_t)p->prof_count * kProfEventsPerEval + k], s);
    }
    void done()
    {
        if (on) ++p->prof_count;
    }
};

// One evaluation of phi (with the self term) and of the force (field = 0) or the
// field -grad phi (field = 1) for charges q at positions x, into phi / frc.  With phi_r / frc_r
// the real space runs on the plan's second stream, concurrently with gridding, the Fourier
// passes and gathering (it needs only the cell-sorted records), and writes there; the caller
// adds them after this returns (s has waited for them).  Without, it adds into phi / frc on s.
template <typename T>
void run_pass(se1p_plan *p, int n, const double *x, const double *q, double *phi, double *frc, int field,
              int check_neutral, cudaStream_t s, StageMarks *m, double *phi_r = nullptr, double *frc_r = nullptr)
{
    const int fl = field ? 2 : 0;
    if (m) m->begin(SE1P_STAGE_PACK, s);
    launch_pack<T>(p, n, x, q, s, check_neutral);
    launch_sort_scatter<T>(p, n, s);
    if (m) m->end(SE1P_STAGE_PACK, s);
    const bool real = p->geo.rc > 0;
    const bool side = real && phi_r && frc_r;
    if (side) {
        cudaEventRecord(p->ev_fork, s);
        cudaStreamWaitEvent(p->s_real, p->ev_fork, 0);
        if (m) m->begin(SE1P_STAGE_REAL, p->s_real);
        launch_real_space<T>(p, n, p->b.cell_key, phi_r, frc_r, fl, p->s_real);
        if (m) m->end(SE1P_STAGE_REAL, p->s_real);
        cudaEventRecord(p->ev_join, p->s_real);
    }
    if (m) m->begin(SE1P_STAGE_SPREAD, s);
    launch_spread<T>(p, s);
    if (m) m->end(SE1P_STAGE_SPREAD, s);
    if (m) m->begin(SE1P_STAGE_FOURIER, s);
    if (p->per3) launch_fold<T>(p, s);
    launch_fourier<T>(p, s);
    if (p->per3) launch_unfold<T>(p, s);
    if (m) m->end(SE1P_STAGE_FOURIER, s);
    if (m) m->begin(SE1P_STAGE_GATHER, s);
    launch_gather<T>(p, n, p->b.grid, phi, frc, 1 | fl | 4, s);
    if (m) m->end(SE1P_STAGE_GATHER, s);
    if (side) {
        cudaStreamWaitEvent(s, p->ev_join, 0);
    } else {
        if (m) m->begin(SE1P_STAGE_REAL, s);
        if (real) launch_real_space<T>(p, n, p->b.cell_key, phi, frc, 1 | fl, s);
        if (m) m->end(SE1P_STAGE_REAL, s);
    }
}

template <typename T>
se1p_status run_eval(se1p_plan *p, int n, const double *x, const double *q, double *phi, double *frc,
                     double *energy, cudaStream_t s)
{
    StageMarks m(p);
    // the real space writes phi2 / frc2 (free outside the adjoint) and the finalisation adds them;
    // profiling mode 2 runs it in sequence with the grid path instead
    const bool real = p->geo.rc > 0 && p->profiling != 2;
    run_pass<T>(p, n, x, q, p->b.phi_int, p->b.frc_int, 0, 1, s, &m, real ? p->b.phi2 : nullptr,
                real ? p->b.frc2 : nullptr);
    m.begin(SE1P_STAGE_FINAL, s);
    launch_finalize(p, n, phi, frc, energy, s, real ? p->b.phi2 : nullptr, real ? p->b.frc2 : nullptr);
    m.end(SE1P_STAGE_FINAL, s);
    m.done();
    return check_launch();
}

template <typename T>
se1p_status run_vjp(se1p_plan *p, int n, const double *x, const double *q, const double *v, double *grad_x,
                    double *grad_q, cudaStream_t s)
{
    run_pass<T>(p, n, x, q, p->b.phi2, p->b.frc2, 1, 1, s, nullptr);      // E[q]
    run_pass<T>(p, n, x, v, p->b.phi_int, p->b.frc_int, 1, 0, s, nullptr);  // phi[v], E[v]
    launch_vjp_combine(n, q, v, p->b.frc2, p->b.phi_int, p->b.frc_int, grad_x, grad_q, s);
    return check_launch();
}

void destroy_events(se1p_plan *p)
{
    for (cudaEvent_t e : p->prof_events) cudaEventDestroy(e);
    p->prof_events.clear();
    p->prof_count = 0;
}

se1p_status flags_to_status(int f)
{
    if (f & FLAG_NAN) return SE1P_ERR_NAN;
    if (f & FLAG_OUT_OF_BOX) return SE1P_ERR_OUT_OF_BOX;
    if (f & FLAG_NOT_NEUTRAL) return SE1P_ERR_NOT_NEUTRAL;
    if (f & FLAG_CAPACITY) return SE1P_ERR_CAPACITY;
    if (f & FLAG_TIMEOUT) return SE1P_ERR_TIMEOUT;
    return SE1P_OK;
}

bool bad_n(const se1p_plan *p, int n) { return n < 0 || n > p->n_max; }

// Real-space cells per cutoff length, from the expected neighbours of a particle within rc at uniform
// density (n_max over the box): finer cells pay where cells are full, coarser ones where they are
// sparse.  Measured (real space alone, FP32): ~1400 neighbours (N = 10^5 in the unit box, rc = 0.15;
// and 2 x 10^5 clustered charges) 0.835 / 16.7 ms with rc / 3 against 0.926 / 18.9 with rc / 2;
// ~380 (N = 10^6 in [1, 1, 8], rc = 0.09) 3.42 ms with rc / 3 against 2.92 with rc / 2 (cells of rc: 3.76), and
// 64 systems of ~230 gained 1.8 % with rc / 2.
constexpr double kCellsDenseNeighbours = 800.0;

// The spread grid holds unnormalised windows; this factor turns it into Eq. 3.4's grid.
double window_norm3(const se1p_plan *p) { return p->geo.wnorm_xy * p->geo.wnorm_xy * p->geo.wnorm_z; }

}  // namespace

extern "C" {

const char *se1p_status_string(se1p_status st)
{
    switch (st) {
    case SE1P_OK: return "SE1P_OK";
    case SE1P_ERR_INVALID_ARG: return "SE1P_ERR_INVALID_ARG";
    case SE1P_ERR_NOT_NEUTRAL: return "SE1P_ERR_NOT_NEUTRAL";
    case SE1P_ERR_OUT_OF_BOX: return "SE1P_ERR_OUT_OF_BOX";
    case SE1P_ERR_ALLOC: return "SE1P_ERR_ALLOC";
    case SE1P_ERR_CUDA: return "SE1P_ERR_CUDA";
    case SE1P_ERR_TIMEOUT: return "SE1P_ERR_TIMEOUT";
    case SE1P_ERR_NAN: return "SE1P_ERR_NAN";
    case SE1P_ERR_CAPACITY: return "SE1P_ERR_CAPACITY";
    }
    return "SE1P_ERR_UNKNOWN";
}

se1p_status se1p_plan_create(const se1p_params *prm, int n_max, se1p_plan **out)
{
    if (!out) return SE1P_ERR_INVALID_ARG;
    *out = nullptr;
    if (!prm || n_max < 0) return SE1P_ERR_INVALID_ARG;
    const se1p_params &P = *prm;
    for (int i = 0; i < 3; ++i)
        if (!(P.L[i] > 0.0) || !isfinite(P.L[i]) || P.M[i] < 1) return SE1P_ERR_INVALID_ARG;
    if (P.L[0] != P.L[1] || P.M[0] != P.M[1]) return SE1P_ERR_INVALID_ARG;
    if (!(P.xi > 0.0) || !isfinite(P.xi)) return SE1P_ERR_INVALID_ARG;
    if (P.P < 2 || P.P > 32 || P.P > P.M[2] || P.P > P.M[0]) return SE1P_ERR_INVALID_ARG;
    if (P.precision != SE1P_FP64 && P.precision != SE1P_MIXED) return SE1P_ERR_INVALID_ARG;
    if (P.flags != 0 && P.flags != SE1P_FLAG_TRIPLY_PERIODIC) return SE1P_ERR_INVALID_ARG;
    const bool per3 = P.flags == SE1P_FLAG_TRIPLY_PERIODIC;
    if (per3 && ((P.P & 1) || !is_smooth(P.M[0]) || (P.rc > 0.0 && P.rc > P.L[0]))) return SE1P_ERR_INVALID_ARG;
    if (!is_smooth(P.M[2])) return SE1P_ERR_INVALID_ARG;
    if (P.rc > 0.0 && (!isfinite(P.rc) || P.rc > P.L[2])) return SE1P_ERR_INVALID_ARG;
    if (P.Mt < 0 || P.n0 < 0 || P.nI < 0) return SE1P_ERR_INVALID_ARG;

    se1p_plan *p = new (std::nothrow) se1p_plan();
    if (!p) return SE1P_ERR_ALLOC;
    p->prm = P;
    p->n_max = n_max;
    p->precision = P.precision;
    cudaGetDevice(&p->device);

    const double tol = P.tol > 0.0 ? P.tol : 1e-10;
    p->M3 = P.M[2];
    p->per3 = per3;
    if (per3) {
        // gridding on the extended grid M + P (a multiple of 4, so that gathering can use 16-byte
        // row vectors), transforms on the periodic grid M: no padding anywhere
        p->Mt = (P.M[0] + P.P + 3) / 4 * 4;
        p->Mf = P.M[0];
    } else {
        p->Mt = P.Mt > 0 ? P.Mt : next_smooth(P.M[0] + P.P);
        if (p->Mt < P.M[0] + P.P || !is_smooth(p->Mt)) { delete p; return SE1P_ERR_INVALID_ARG; }
        p->Mf = p->Mt;
    }
    const double s0 = P.s0 > 0.0 ? P.s0 : 2.0 * sqrt(2.0);
    p->n0 = per3 ? p->Mf : (P.n0 > 0 ? P.n0 : next_smooth((long)ceil(s0 * p->Mt - 1e-9)));
    double sl = P.sl;
    if (!(sl > 0.0)) {  // e^{-2 pi sl} < tol (Eq. 4.8)
        sl = -log(tol) / (2.0 * kPi);
        if (sl < 1.0) sl = 1.0;
    }
    p->nI = per3 ? p->Mf : (P.nI > 0 ? P.nI : next_smooth((long)ceil(sl * p->Mt - 1e-9)));
    p->nl = per3 ? 0 : (P.nl >= 0 ? P.nl : (P.M[2] / 10 > 1 ? (int)lround(P.M[2] / 10.0) : 1));  // M ~ 10 nl (Eq. 4.9)
    if (p->n0 < p->Mf || p->nI < p->Mf || !is_smooth(p->n0) || !is_smooth(p->nI)) { delete p; return SE1P_ERR_INVALID_ARG; }
    p->K3 = p->M3 / 2 + 1;

    Geo &g = p->geo;
    g.M3 = p->M3;
    g.Mt = p->Mt;
    g.P = P.P;
    g.K3 = p->K3;
    g.c = (P.P & 1) ? (P.P - 1) / 2 : P.P / 2;
    g.nbx = (p->Mt - P.P) / kBin + 1;
    g.nby = g.nbx;
    g.nbz = (p->M3 + kBin - 1) / kBin;
    g.nbins = g.nbx * g.nby * g.nbz;
    for (int i = 0; i < 3; ++i) g.L[i] = P.L[i];
    g.h = P.L[0] / P.M[0];
    g.hz = P.L[2] / P.M[2];
    g.off = P.P * g.h / 2.0;
    g.inv_h = 1.0 / g.h;
    g.inv_hz = 1.0 / g.hz;
    g.xi = P.xi;
    g.eta = P.P * P.xi * P.xi * g.h * g.h / (kShapeC * kShapeC * kPi);     // Eq. 3.3
    g.etaz = P.P * P.xi * P.xi * g.hz * g.hz / (kShapeC * kShapeC * kPi);
    g.wnorm_xy = sqrt(2.0 * P.xi * P.xi / (kPi * g.eta));
    g.wnorm_z = sqrt(2.0 * P.xi * P.xi / (kPi * g.etaz));
    g.alpha_xy = 2.0 * P.xi * P.xi * g.h * g.h / g.eta;
    g.alpha_z = 2.0 * P.xi * P.xi * g.hz * g.hz / g.etaz;
    g.per3 = per3 ? 1 : 0;
    g.rc = P.rc > 0.0 ? P.rc : 0.0;
    g.rc2 = g.rc * g.rc;
    if (g.rc > 0.0) {
        // cells of edge >= rc / 3 (dense) or rc / 2 (stencil of +-3 or +-2 cells), at most 2^22 cells
        const double neighbours = (double)(n_max > 0 ? n_max : 1) / (P.L[0] * P.L[1] * P.L[2]) * 4.0 / 3.0 * kPi *
                                  g.rc * g.rc * g.rc;
        const double ce = g.rc / (neighbours >= kCellsDenseNeighbours ? 3.0 : 2.0);
        g.ncx = (int)fmin(fmax(floor(P.L[0] / ce), 1.0), 1024.0);
        g.ncy = (int)fmin(fmax(floor(P.L[1] / ce), 1.0), 1024.0);
        g.ncz = (int)fmin(fmax(floor(P.L[2] / ce), 1.0), 8192.0);
        while ((long)g.ncx * g.ncy * g.ncz > (1L << 22)) {
            if (g.ncz >= g.ncx) g.ncz = (g.ncz + 1) / 2;
            else { g.ncx = (g.ncx + 1) / 2; g.ncy = (g.ncy + 1) / 2; }
        }
    } else {
        g.ncx = g.ncy = g.ncz = 1;
    }
    g.ncells = g.ncx * g.ncy * g.ncz;
    g.cs[0] = P.L[0] / g.ncx;
    g.cs[1] = P.L[1] / g.ncy;
    g.cs[2] = P.L[2] / g.ncz;
    int nIm = 0;
    for (int k = 1; k < p->K3 && !per3; ++k)
        if (k * P.L[0] / P.L[2] <= p->nl * (1.0 + 1e-12)) nIm = k;
    g.nIm = nIm;

    // slab classes: k3 = 0 (FP64), I (nI), J (Mt)
    p->cls[0].ns = p->n0; p->cls[0].kfirst = 0; p->cls[0].count = 1;
    p->cls[1].ns = p->nI; p->cls[1].kfirst = 1; p->cls[1].count = nIm;
    p->cls[2].ns = p->Mf; p->cls[2].kfirst = 1 + nIm; p->cls[2].count = p->K3 - 1 - nIm;
    bool fft_ok = make_fft(p->M3, p->fd_z);
    for (int c = 0; c < 3; ++c) fft_ok = fft_ok && make_fft(p->cls[c].ns, p->cls[c].fd);
    if (!fft_ok) { delete p; return SE1P_ERR_INVALID_ARG; }

    const bool mixed = P.precision == SE1P_MIXED;
    const size_t cT = mixed ? sizeof(Cx<float>) : sizeof(Cx<double>);
    // pencils per CTA: as many as shared memory allows, but few enough that each
    // pass launches at least ~2 CTAs per SM (152 SMs)
    const long min_ctas = 2 * 152;
    auto shrink = [&](int v, long units) {
        while (v > 1 && (units + v - 1) / v < min_ctas) v >>= 1;
        return v;
    };
    // z passes: a CTA holds xb_z complex pencils of M3 points (twice, for the Stockham passes); with Mt
    // even each complex pencil carries two real ones
    p->xb_z = shrink(pow2_fit(2 * (size_t)p->M3 * cT, 32), (long)(p->Mf + 1) / 2 * p->Mf);
    for (int c = 0; c < 3; ++c) {
        const size_t cc = c == 0 ? sizeof(Cx<double>) : cT;
        SlabClass &C = p->cls[c];
        C.rb = shrink(pow2_fit(2 * (size_t)C.ns * cc, 16), (long)C.count * p->Mf);
        C.xb = shrink(pow2_fit(2 * (size_t)C.ns * cc, 32), (long)C.count * C.ns);
    }
    if (2 * (size_t)p->M3 * cT * p->xb_z > 200 * 1024) { delete p; return SE1P_ERR_INVALID_ARG; }
    for (int c = 0; c < 3; ++c) {
        const size_t cc = c == 0 ? sizeof(Cx<double>) : cT;
        if (2 * (size_t)p->cls[c].ns * cc > 200 * 1024) { delete p; return SE1P_ERR_INVALID_ARG; }
    }

    Alloc A{p};
    if (const char *e = getenv("SE1P_TEST_FAIL_ALLOC")) A.fail_at = atoi(e);
    // polls of the bounded device waits; SE1P_TEST_SPIN_LIMIT (tests only) makes them give up early
    if (const char *e = getenv("SE1P_TEST_SPIN_LIMIT")) p->spin_limit = atoll(e);
    se1p_status st = mixed ? alloc_particles<float>(p, A) : alloc_particles<double>(p, A);
    if (st == SE1P_OK) st = mixed ? build_tables<float>(p, A) : build_tables<double>(p, A);
    if (st != SE1P_OK) { free_all(p); delete p; return st; }
    int cfg = mixed ? configure_fourier_kernels<float>(p) : configure_fourier_kernels<double>(p);
    if (cfg == 0) cfg = mixed ? configure_particle_kernels<float>(p) : configure_particle_kernels<double>(p);
    if (cfg != 0) { cudaGetLastError(); free_all(p); delete p; return SE1P_ERR_CUDA; }
    bool streams_ok = cudaStreamCreateWithFlags(&p->s_real, cudaStreamNonBlocking) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < 2; ++i)
        streams_ok = streams_ok && cudaStreamCreateWithFlags(&p->s_f[i], cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; i < 3; ++i)
        streams_ok = streams_ok && cudaEventCreateWithFlags(&p->ev_f[i], cudaEventDisableTiming) == cudaSuccess;
    if (!streams_ok) {
        cudaGetLastError();
        free_all(p);
        delete p;
        return SE1P_ERR_CUDA;
    }
    if (per3) launch_k3zero_table_3p(p, 0);
    else launch_vico_table(p, 0);
    if (mixed) launch_symbol_tables<float>(p, 0);
    else launch_symbol_tables<double>(p, 0);
    if (cudaDeviceSynchronize() != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_all(p);
        delete p;
        return SE1P_ERR_CUDA;
    }
    *out = p;
    return SE1P_OK;
}

se1p_status se1p_plan_destroy(se1p_plan *p)
{
    if (!p) return SE1P_OK;
    cudaDeviceSynchronize();
    destroy_events(p);
    free_all(p);
    delete p;
    return SE1P_OK;
}

se1p_status se1p_plan_get_info(const se1p_plan *p, se1p_plan_info *info)
{
    if (!p || !info) return SE1P_ERR_INVALID_ARG;
    memset(info, 0, sizeof(*info));
    info->Mt = p->Mt;
    info->M3 = p->M3;
    info->n0 = p->n0;
    info->nI = p->nI;
    info->nl = p->nl;
    info->n_I_modes = p->geo.nIm;
    info->P = p->geo.P;
    info->precision = p->precision;
    info->h = p->geo.h;
    info->hz = p->geo.hz;
    info->eta = p->geo.eta;
    info->etaz = p->geo.etaz;
    info->R = sqrt(2.0) * p->Mt * p->geo.h;
    info->cells[0] = p->geo.ncx;
    info->cells[1] = p->geo.ncy;
    info->cells[2] = p->geo.ncz;
    info->features = p->tma_zfwd ? 1 : 0;
    info->workspace_bytes = p->bytes;
    return SE1P_OK;
}

se1p_status se1p_eval(se1p_plan *p, int n, const double *x, const double *q, double *phi, double *force,
                      double *energy, void *stream)
{
    if (!p || bad_n(p, n) || (n > 0 && (!x || !q))) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        if (energy) cudaMemsetAsync(energy, 0, sizeof(double), s);
        return check_launch();
    }
    return p->precision == SE1P_MIXED ? run_eval<float>(p, n, x, q, phi, force, energy, s)
                                      : run_eval<double>(p, n, x, q, phi, force, energy, s);
}

se1p_status se1p_plan_set_profiling(se1p_plan *p, int enable)
{
    if (!p || enable < 0 || enable > 2) return SE1P_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return SE1P_ERR_CUDA;
    destroy_events(p);
    p->profiling = 0;
    if (!enable) return SE1P_OK;
    p->prof_events.resize((size_t)kProfMaxEvals * kProfEventsPerEval);
    for (auto &e : p->prof_events) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            e = nullptr;
            cudaGetLastError();
            destroy_events(p);
            return SE1P_ERR_CUDA;
        }
    }
    p->profiling = enable;
    return SE1P_OK;
}

se1p_status se1p_plan_stage_times(se1p_plan *p, double *ms, int *n_evals)
{
    if (!p || !ms) return SE1P_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return SE1P_ERR_CUDA;
    for (int st = 0; st < SE1P_NUM_STAGES; ++st) ms[st] = 0.0;
    for (int e = 0; e < p->prof_count; ++e) {
        for (int st = 0; st < SE1P_NUM_STAGES; ++st) {
            float t = 0.f;
            cudaEvent_t a = p->prof_events[(size_t)e * kProfEventsPerEval + 2 * st];
            cudaEvent_t b = p->prof_events[(size_t)e * kProfEventsPerEval + 2 * st + 1];
            if (cudaEventElapsedTime(&t, a, b) != cudaSuccess) return SE1P_ERR_CUDA;
            ms[st] += t;
        }
    }
    if (n_evals) *n_evals = p->prof_count;
    p->prof_count = 0;
    return SE1P_OK;
}

se1p_status se1p_eval_vjp(se1p_plan *p, int n, const double *x, const double *q, const double *v_phi,
                          double *grad_x, double *grad_q, void *stream)
{
    if (!p || bad_n(p, n) || (n > 0 && (!x || !q || !v_phi))) return SE1P_ERR_INVALID_ARG;
    if (n == 0) return SE1P_OK;
    cudaStream_t s = (cudaStream_t)stream;
    return p->precision == SE1P_MIXED ? run_vjp<float>(p, n, x, q, v_phi, grad_x, grad_q, s)
                                      : run_vjp<double>(p, n, x, q, v_phi, grad_x, grad_q, s);
}

se1p_status se1p_plan_sync_status(se1p_plan *p, void *stream)
{
    if (!p) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SE1P_ERR_CUDA;
    int f = 0;
    if (cudaMemcpy(&f, p->b.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SE1P_ERR_CUDA;
    cudaMemset(p->b.status, 0, sizeof(int));
    if (cudaDeviceSynchronize() != cudaSuccess) return SE1P_ERR_CUDA;
    return flags_to_status(f);
}

se1p_status se1p_eval_host(se1p_plan *p, int n, const double *x, const double *q, double *phi, double *force,
                           double *energy, void *stream)
{
    if (!p || bad_n(p, n) || (n > 0 && (!x || !q))) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n > 0) {
        cudaMemcpyAsync(p->b.hx, x, sizeof(double) * 3 * (size_t)n, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(p->b.hq, q, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, s);
    }
    se1p_status st = se1p_eval(p, n, p->b.hx, p->b.hq, phi ? p->b.hphi : nullptr, force ? p->b.hfrc : nullptr,
                               energy ? p->b.hen : nullptr, stream);
    if (st != SE1P_OK) return st;
    if (phi && n > 0) cudaMemcpyAsync(phi, p->b.hphi, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (force && n > 0) cudaMemcpyAsync(force, p->b.hfrc, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost, s);
    if (energy) cudaMemcpyAsync(energy, p->b.hen, sizeof(double), cudaMemcpyDeviceToHost, s);
    // the status word travels with the outputs and is cleared on the stream: one blocking sync
    cudaMemcpyAsync(p->b.hstatus, p->b.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaMemsetAsync(p->b.status, 0, sizeof(int), s);
    if (check_launch() != SE1P_OK) return SE1P_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SE1P_ERR_CUDA;
    return flags_to_status(*p->b.hstatus);
}

se1p_status se1p_spread(se1p_plan *p, int n, const double *x, const double *q, double *grid, void *stream)
{
    if (!p || p->per3 || bad_n(p, n) || !grid || (n > 0 && (!x || !q))) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->precision == SE1P_MIXED) {
        launch_pack<float>(p, n, x, q, s);
        launch_sort_scatter<float>(p, n, s);
        launch_spread<float>(p, s);
        launch_grid_to_double<float>(p, p->b.grid, grid, window_norm3(p), s);
    } else {
        launch_pack<double>(p, n, x, q, s);
        launch_sort_scatter<double>(p, n, s);
        launch_spread<double>(p, s);
        launch_grid_to_double<double>(p, p->b.grid, grid, window_norm3(p), s);
    }
    return check_launch();
}

se1p_status se1p_fourier(se1p_plan *p, const double *grid_in, double *grid_out, void *stream)
{
    if (!p || p->per3 || !grid_in || !grid_out) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (p->precision == SE1P_MIXED) {
        launch_grid_from_double<float>(p, grid_in, p->b.grid, s);
        launch_fourier<float>(p, s);
        launch_grid_to_double<float>(p, p->b.grid, grid_out, 1.0, s);
    } else {
        launch_grid_from_double<double>(p, grid_in, p->b.grid, s);
        launch_fourier<double>(p, s);
        launch_grid_to_double<double>(p, p->b.grid, grid_out, 1.0, s);
    }
    return check_launch();
}

se1p_status se1p_gather(se1p_plan *p, int n, const double *x, const double *q, const double *grid, double *phi,
                        double *force, void *stream)
{
    if (!p || p->per3 || bad_n(p, n) || !grid || (n > 0 && (!x || !q))) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return SE1P_OK;
    if (p->precision == SE1P_MIXED) {
        launch_pack<float>(p, n, x, q, s);
        launch_sort_scatter<float>(p, n, s);
        launch_grid_from_double<float>(p, grid, p->b.grid, s);
        launch_gather<float>(p, n, p->b.grid, p->b.phi_int, p->b.frc_int, 0, s);
    } else {
        launch_pack<double>(p, n, x, q, s);
        launch_sort_scatter<double>(p, n, s);
        launch_grid_from_double<double>(p, grid, p->b.grid, s);
        launch_gather<double>(p, n, p->b.grid, p->b.phi_int, p->b.frc_int, 0, s);
    }
    launch_finalize(p, n, phi, force, nullptr, s);
    return check_launch();
}

se1p_status se1p_real_space(se1p_plan *p, int n, const double *x, const double *q, double *phi, double *force,
                            void *stream)
{
    if (!p || bad_n(p, n) || (n > 0 && (!x || !q)) || !(p->geo.rc > 0.0)) return SE1P_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return SE1P_OK;
    if (p->precision == SE1P_MIXED) {
        launch_pack<float>(p, n, x, q, s);
        launch_sort_scatter<float>(p, n, s);
        launch_real_space<float>(p, n, p->b.cell_key, p->b.phi_int, p->b.frc_int, 0, s);
    } else {
        launch_pack<double>(p, n, x, q, s);
        launch_sort_scatter<double>(p, n, s);
        launch_real_space<double>(p, n, p->b.cell_key, p->b.phi_int, p->b.frc_int, 0, s);
    }
    launch_finalize(p, n, phi, force, nullptr, s);
    return check_launch();
}

}  // extern "C"
