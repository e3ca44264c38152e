// Host-side plan object and kernel launchers of libse1p (internal).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

#include "se1p_internal.cuh"

namespace se1p {

// One class of k3 slabs sharing a padded 2-D size (k3 = 0, the set I, the set J).
struct SlabClass {
    int ns = 0;       // padded 2-D size
    int kfirst = 0;   // first k3 index of the class
    int count = 0;    // number of k3 indices
    FftDesc fd{};     // FFT of length ns
    void *tw = nullptr;     // twiddles (Cx<T>, or Cx<double> for class 0)
    void *rows = nullptr;   // [count][Mt][ns] complex work rows
    void *sym = nullptr;    // classes 1, 2: scaling symbol incl. normalisation, [count][ns][ns] (T)
    int rb = 1;             // rows per CTA in the x passes
    int xb = 1;             // columns per CTA in the y pass
};

struct Buffers {
    void *grid = nullptr;        // T, M3 x Mt x Mt points in x-blocks (gidx)
    void *gridf = nullptr;       // T, M3 x Mf x Mf periodic grid of the FFTs (triply periodic plans; else = grid)
    void *zspec = nullptr;       // Cx<T> [K3][Mt][Mt]  (k3 = 0 entry unused)
    double *slab0_in = nullptr;  // k3 = 0 coefficient of H, [Mt][Mt]
    double *slab0_out = nullptr; // k3 = 0 coefficient of Ht, [Mt][Mt]
    double *sym0 = nullptr;      // k3 = 0 scaling incl. normalisation, [n0][n0]
    void *tw_z = nullptr;        // Cx<T> [M3]
    double *xyzq = nullptr;      // sanitised caller-order particles [n_max][4]
    int *bin_key = nullptr, *cell_key = nullptr;
    int *counts = nullptr;       // [nbins + ncells]
    int *starts = nullptr;       // [nbins + 1 + ncells + 1]
    int *cursors = nullptr;      // [nbins + ncells]
    int *scan_tmp = nullptr;     // block offsets of the multi-block cell scan [kScanTmp]
    int *gchunk = nullptr;       // [kGatherChunks] cursor of each chunk sequence of the gather's handout
    void *parts = nullptr;       // PartRec<T> [n_max]
    void *wts = nullptr;         // T [n_max][3][P]
    void *cells = nullptr;       // CellRec<T> [n_max]
    double *phi_int = nullptr;   // [n_max]
    double *frc_int = nullptr;   // [n_max][3]
    double *phi2 = nullptr;      // [n_max]     second evaluation of the adjoint
    double *frc2 = nullptr;      // [n_max][3]
    double *rsum = nullptr;      // [4][n_max] FP64 real-space sums (phi, field) in cell order
    double *sums = nullptr;      // [2] sum q, sum |q|
    double *epart = nullptr;     // [kEnergyBlocks]
    int *status = nullptr;
    double *hx = nullptr, *hq = nullptr, *hphi = nullptr, *hfrc = nullptr, *hen = nullptr;  // host staging
    int *hstatus = nullptr;  // page-locked copy of the status word (host entry point)
};

constexpr int kEnergyBlocks = 256;
// chunk sequences of the gather's handout at most (one per SM)
constexpr int kGatherChunks = 256;

}  // namespace se1p

struct se1p_plan {
    se1p_params prm{};
    se1p::Geo geo{};
    int n_max = 0;
    int precision = 0;
    int device = 0;
    int nsm = 1;  // SMs of the device
    int gather_ctas = 1;  // resident CTAs of the gather kernels (SMs x CTAs per SM of the largest instance)
    int Mt = 0, M3 = 0, K3 = 0, n0 = 0, nI = 0, nl = 0;
    // free-axis size of the transformed grid: Mt for SE1P; M for triply periodic plans, whose gridding
    // runs on the Mt = M + P extended grid and is folded onto the M-periodic grid before the FFTs
    int Mf = 0;
    bool per3 = false;
    se1p::FftDesc fd_z{};
    int xb_z = 1;      // z passes: pencil pairs per CTA (two real pencils as one complex pencil; for odd
                       // Mf the last pencil pairs with the zero padding of the x-blocked grid)
    // z forward pass by bulk tensor copies (tma_zfwd) of zbox-deep boxes; polls of its bounded wait
    CUtensorMap tm_zfwd{};
    bool tma_zfwd = false;
    int tma_zbox = 0;
    long long spin_limit = 1ll << 22;
    se1p::SlabClass cls[3];  // 0: k3 = 0 (FP64 always), 1: I, 2: J
    se1p::Buffers b;
    std::vector<void *> dev_allocs;
    std::vector<void *> host_allocs;
    size_t bytes = 0;
    double norm_k3 = 0;  // 4 pi / M3 (class-specific 1/ns^2 applied in kernels)
    // real space runs on its own stream, concurrently with the grid path (fork / join events)
    cudaStream_t s_real = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // slab classes 0 and 1 of the Fourier passes run on their own streams (fork ev_f[0], joins 1, 2)
    cudaStream_t s_f[2] = {nullptr, nullptr};
    cudaEvent_t ev_f[3] = {nullptr, nullptr, nullptr};
    // per-stage profiling events: [eval][stage][start, end], each on the stream the stage runs on
    int profiling = 0;
    int prof_count = 0;
    std::vector<cudaEvent_t> prof_events;
};

namespace se1p {

// ---- se1p_particles.cu
template <typename T>
void launch_pack(se1p_plan *p, int n, const double *x, const double *q, cudaStream_t s, int check_neutral = 1);
template <typename T> void launch_sort_scatter(se1p_plan *p, int n, cudaStream_t s);
template <typename T> void launch_spread(se1p_plan *p, cudaStream_t s);
// flags: bit 0 adds the self term, bit 1 writes the field -grad phi instead of the force
template <typename T> void launch_gather(se1p_plan *p, int n, const void *grid, double *phi, double *frc,
                                         int flags, cudaStream_t s);
void launch_vjp_combine(int n, const double *q, const double *v, const double *Eq, const double *phiv,
                        const double *Ev, double *grad_x, double *grad_q, cudaStream_t s);
void launch_finalize(se1p_plan *p, int n, double *phi, double *frc, double *energy, cudaStream_t s,
                     const double *phi_add = nullptr, const double *frc_add = nullptr);
template <typename T>
void launch_grid_to_double(se1p_plan *p, const void *src, double *dst, double scale, cudaStream_t s);
template <typename T> void launch_grid_from_double(se1p_plan *p, const double *src, void *dst, cudaStream_t s);
template <typename T> int configure_particle_kernels(se1p_plan *p);
// triply periodic plans: fold the extended spread grid onto the periodic grid, and back
template <typename T> void launch_fold(se1p_plan *p, cudaStream_t s);
template <typename T> void launch_unfold(se1p_plan *p, cudaStream_t s);

// ---- se1p_fourier.cu
template <typename T> void launch_fourier(se1p_plan *p, cudaStream_t s);
template <typename T> int configure_fourier_kernels(se1p_plan *p);
void launch_vico_table(se1p_plan *p, cudaStream_t s);
void launch_k3zero_table_3p(se1p_plan *p, cudaStream_t s);
template <typename T> void launch_symbol_tables(se1p_plan *p, cudaStream_t s);

// ---- se1p_real.cu
// flags: bit 0 accumulates into phi/frc (else they are overwritten), bit 1 writes the field
template <typename T> void launch_real_space(se1p_plan *p, int n, const int *cell_key, double *phi, double *frc,
                                             int flags, cudaStream_t s);

}  // namespace se1p
