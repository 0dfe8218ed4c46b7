// Internal declarations of the to3d CUDA library (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>

#include "../../include/to3d.h"

namespace to3d {

// ---------------------------------------------------------------- geometry
struct Grid {
    int nelx, nely, nelz;     // elements per axis
    int nx, ny, nz;           // nodes per axis (= elements + 1)
    long long nel, nnode;
};

__host__ __device__ inline long long elem_id(const Grid& g, int i, int j, int k) {
    return (long long)i + (long long)g.nelx * ((long long)j + (long long)g.nely * k);
}
__host__ __device__ inline long long node_id(const Grid& g, int i, int j, int k) {
    return (long long)i + (long long)g.nx * ((long long)j + (long long)g.ny * k);
}

// Element stiffness for unit modulus, passed by value to kernels (it lives in
// the kernel parameter constant bank, so each context may use its own nu).
struct KE64 { double v[576]; };
// Integer split KE = c_lam * A_lam + c_mu * A_mu (A_lam, A_mu integer-valued).
struct KESplit { float a_lam[576]; float a_mu[576]; double c_lam, c_mu; };

// Filter stencil: integer offsets and weights rmin - |d| > 0.
constexpr int kMaxStencil = 1200;
struct Stencil {
    int n;
    int radius;
    int off[kMaxStencil];      // packed (di+16) | (dj+16) << 8 | (dk+16) << 16
    double w[kMaxStencil];
};

// ---------------------------------------------------------------- scalars
// Device-resident solver / OC state, so loops need no host round trip.
struct SolverScalars {
    double rz, rz_new, pq, rr, alpha, beta;
    double zcoef;             // coefficient of M^-1 r in the next direction (1 except
                              // right after a residual replacement)
    double fnorm2, tol2;
    double rr_true;
    int it, done, status, maxit;
    int restarts, pad0, pad1, pad2;
};

struct OCScalars {
    double l1, l2, lmid, tol, target;
    double cand[64];          // candidate lambdas of the current pass (tree order)
    int ncand, levels, halvings, done;
    int status, maxhalv, pad0, pad1;
    double volume, change;
};

// Grid-wide deterministic reductions: per-block partials, last block sums.
struct Reducer {
    double* partials = nullptr;   // [kMaxReduceVals][kMaxBlocks]
    unsigned int* counter = nullptr;
};
constexpr int kMaxReduceVals = 64;
constexpr int kMaxBlocks = 1 << 16;

const char* status_name(to3d_status s);

}  // namespace to3d

// ---------------------------------------------------------------- context
struct to3d_ctx {
    to3d_params prm;
    to3d::Grid g;
    cudaStream_t stream = nullptr;        // caller's stream
    cudaStream_t cap_stream = nullptr;    // private stream used only for graph capture
    int device = 0;
    std::string err;
    long long launches = 0;
    int iter = 0;
    bool trace = false;
    bool have_u = false;
    int pcg_its_est = 0;           // iterations of the last FP64 Jacobi-PCG solve (0: none yet)
    const double* xop = nullptr;   // densities the operator was last prepared for (device)
    double* xphys = nullptr;       // filtered densities of the density-filter OC step
    bool have_dinv = false;

    to3d::KE64 ke;                        // unit-modulus element stiffness
    to3d::KESplit kes;
    to3d::Stencil* st = nullptr;          // host copy of the filter stencil

    // design / element arrays [nel]
    double *x = nullptr, *xnew = nullptr, *E = nullptr;
    float* E32 = nullptr;                 // FP32 moduli, x extent padded to pex (pads 0)
    double *ce = nullptr, *dc = nullptr, *dcf = nullptr, *Hs = nullptr;
    double *ocq = nullptr, *oclo = nullptr, *ochi = nullptr;
    float* ocs = nullptr;    // q, lo, hi as FP32 (hi, lo) pairs: [nel][6] (OC passes)
    uint8_t* passive = nullptr;
    // node arrays
    uint8_t* nodemask = nullptr;          // [N] bit c set = dof c clamped
    double* dinv = nullptr;               // [N] 1/diag (same for the 3 dofs), 0 if all clamped
    float* dinv32 = nullptr;
    // dof arrays [3N]
    double *f = nullptr, *ftmp = nullptr, *u = nullptr, *r = nullptr, *p = nullptr, *q = nullptr,
           *tmp = nullptr;
    float *d32 = nullptr, *r32 = nullptr, *p32a = nullptr, *p32b = nullptr, *q32 = nullptr;
    // scratch for API calls with host pointers
    void* stage = nullptr;
    size_t stage_bytes = 0, stage_slot = 0;
    int* dev_err = nullptr;               // device error word of the tensor-core kernels
    // padded structure-of-arrays layout of the FP32 inner-solve vectors:
    // component c of node (i,j,k) at c*vol + i + px*(j + ny*k), px = nx rounded up to 4
    int px = 0;
    long long vol = 0;
    uint8_t* maskp = nullptr;             // [vol] clamp bits per padded node (pads: 0xff)
    int pex = 0;                          // x extent of E32, nelx rounded up to 4
    CUtensorMap tm_r, tm_pa, tm_pb, tm_d, tm_e;   // TMA descriptors of r32, p32a, p32b, dinv32, E32
    uint8_t* tcB = nullptr;               // tensor-core B operand images (BF16 then FP16)
    bool tc_split = false;                // B = [A_lam; A_mu] (N = 48) instead of one matrix
    float tc_cscale = 1.f;                // scale of the combined integer B
    double tc_cscale_d = 1.0;             // the same scale in FP64
    double tc_bmax = 0.0;                 // max |B| of the combined integer B
    int tc_lz = 20;                       // node layers per z segment of a tile
    int tc_grid = 608;                    // persistent CTAs
    long long ndesign = 0;                // number of design (non-passive) elements

    to3d::Reducer red;
    to3d::SolverScalars* ss = nullptr;    // device
    to3d::SolverScalars* ss_h = nullptr;  // pinned host mirror
    to3d::OCScalars* os = nullptr;
    to3d::OCScalars* os_h = nullptr;
    double* misc = nullptr;               // device scalars: [0] compliance, [1] volume, [2] change
    double* misc_h = nullptr;
    double fnorm = 0.0;

    cudaEvent_t ev[8] = {};
    // sampled per-launch timing of the dominant kernels (event-record nodes
    // inside the captured solver chunks): [0] tensor-core matvec, [1] FP64 matvec
    static constexpr int kTimedSlots = 16;
    cudaEvent_t kev[2][2 * kTimedSlots] = {};
    int kslot_iter[2][kTimedSlots] = {};     // chunk-local iteration of each sample
    int kslots[2] = {0, 0};
    double kt_ms[2] = {0.0, 0.0};
    long long kt_n[2] = {0, 0};
    cudaGraphExec_t g_pcg64 = nullptr;    // chunk of FP64 PCG iterations
    cudaGraphExec_t g_pcg32 = nullptr;    // chunk of inner FP32 PCG iterations
    int g_pcg32_prec = -1;
    int chunk = 32;
    cudaGraphExec_t g_iter = nullptr;     // whole OC iteration with device-side loops
    cudaStream_t cap_stream2 = nullptr, cap_stream3 = nullptr;   // nested loop-body captures
    void* dcctl = nullptr;                // device control block of the graph's solver
    void* dcctl_h = nullptr;              // pinned copy of it
    void* cnn = nullptr;                  // learned preconditioner (network, workspaces)
    void* mg = nullptr;                   // learned multigrid preconditioner (levels, buffers)
};

// ---------------------------------------------------------------- launchers
namespace to3d {

// error helpers (api.cu)
to3d_status set_err(to3d_ctx* c, to3d_status s, const std::string& msg);
to3d_status cuda_check(to3d_ctx* c, cudaError_t e, const char* what);
to3d_status launch_check(to3d_ctx* c, const char* what);

// matvec64.cu
void launch_matvec64(to3d_ctx* c, cudaStream_t s, const double* E, const double* p, double* y,
                     bool dot_pq);
void launch_diag(to3d_ctx* c, cudaStream_t s, const double* E);
void launch_simp(to3d_ctx* c, cudaStream_t s, const double* x);
void launch_residual64(to3d_ctx* c, cudaStream_t s, const double* f, const double* Ku, double* r,
                       bool to_ss);

// pcg.cu
void launch_pcg64_init(to3d_ctx* c, cudaStream_t s);
void launch_pcg64_iter(to3d_ctx* c, cudaStream_t s, cudaEvent_t ev0 = nullptr,
                       cudaEvent_t ev1 = nullptr);
void launch_pcg32_init(to3d_ctx* c, cudaStream_t s, const double* r64, double scale);
void launch_pcg32_replace(to3d_ctx* c, cudaStream_t s, const double* r64, double scale,
                          const float* p_latest, double delta2, double target2);
void launch_pcg32_iter(to3d_ctx* c, cudaStream_t s, int prec, int parity,
                       cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
void launch_axpy_d32(to3d_ctx* c, cudaStream_t s, double inv_scale);
void launch_norm2(to3d_ctx* c, cudaStream_t s, const double* v, long long n, double* out);
void launch_ss_reset(to3d_ctx* c, cudaStream_t s, double tol2, int maxit);
void launch_ss_segment(to3d_ctx* c, cudaStream_t s, double tol2, int maxit);
inline void launch_fill_zero(to3d_ctx*, cudaStream_t s, void* ptr, size_t bytes) {
    cudaMemsetAsync(ptr, 0, bytes, s);
}
void launch_mask_copy(to3d_ctx* c, cudaStream_t s, const double* src, double* dst);

// matvec_tc.cu
void launch_matvec_tc(to3d_ctx* c, cudaStream_t s, int prec, bool fused, int parity);
// matvec_x64.cu: FP64-accurate K p on the tensor cores (integer slicing)
bool matvec_x64_available(const to3d_ctx* c);
void launch_matvec_x64(to3d_ctx* c, cudaStream_t s, const double* E, const double* p, double* y,
                       bool dot_pq);
// element energies ce_e = u_e^T KE u_e by the same slicing (needs matvec_x64_available)
void launch_energies_x64(to3d_ctx* c, cudaStream_t s, const double* u, double* ce);
void launch_matvec_tc_io(to3d_ctx* c, cudaStream_t s, int prec, bool fused, const CUtensorMap& tr,
                         const CUtensorMap& tp, const CUtensorMap& td, float* p_new, float* q,
                         SolverScalars* ss);
bool encode_vec_map(to3d_ctx* c, CUtensorMap* map, const float* base, int comps);
// time the tensor-core kernel's z-segment lengths once per grid shape and
// precision (cached) and keep the fastest in c->tc_lz (plain form, input
// mapped by tp, output q)
cudaError_t tune_tc_lz(to3d_ctx* c, int prec, const CUtensorMap& tp, float* q, bool set_moduli);
void launch_aos_to_soa(to3d_ctx* c, cudaStream_t s, const float* in, float* out);
void launch_soa_to_aos(to3d_ctx* c, cudaStream_t s, const float* q, const float* p, float* y);
void init_tc_attributes();
bool prepare_tc_operands(to3d_ctx* c);

// element.cu
void launch_check_unit(to3d_ctx* c, cudaStream_t s, const double* x, int* bad);
void launch_pin_passive(to3d_ctx* c, cudaStream_t s, double* x);
void launch_zero_passive(to3d_ctx* c, cudaStream_t s, double* v);
void launch_sensitivity(to3d_ctx* c, cudaStream_t s, const double* x, const double* u,
                        double* ce, double* dc);
void launch_hs(to3d_ctx* c, cudaStream_t s);
void launch_sensitivity_raw(const KE64& ke, const Grid& g, cudaStream_t s, const double* x,
                            const double* u, double penal, double E0, double Emin, double* ce,
                            double* dc, const Reducer& red, double* comp_out);
bool unit_ke(double nu, KE64* out);
// solver helpers shared with the learned-preconditioner code
to3d_status prepare_op(to3d_ctx* c, const double* x);
to3d_status stage_input(to3d_ctx* c, const void* src, size_t bytes, int on_device, size_t slot,
                        const void** out);
to3d_status run_pcg64_iters(to3d_ctx* c, const double* f, int iters);
to3d_status solve64_rtol(to3d_ctx* c, const double* f, double fnorm, double rtol,
                         to3d_solve_info* info);
to3d_status solve64_from_u(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info);
void destroy_cnn(to3d_ctx* c);
// flexible CG (cnn.cu) with a preconditioner supplied by its owner
struct FcgIO {
    double *z = nullptr, *rprev = nullptr, *dots = nullptr, *dots_h = nullptr;
    // z = M r for the FP64 residual r with |r|^2 = rr
    to3d_status (*apply)(to3d_ctx* c, const double* r, double* z, double rr) = nullptr;
};
to3d_status true_residual64(to3d_ctx* c, const double* f, double fnorm, double* relres);
to3d_status sync_solver_scalars(to3d_ctx* c);
// add the sampled tensor-core kernel durations of a completed chunk that
// covered solver iterations [it0, it1)
void accumulate_tc_times(to3d_ctx* c, int it0, int it1);
void launch_pcg32_update_mode(to3d_ctx* c, cudaStream_t s, const float* p_new, int jacobi_beta);
void launch_dots64(to3d_ctx* c, cudaStream_t s, long long n, const double* a, const double* b,
                   const double* cc, const double* d, double* out_dev);
// mg.cu
void destroy_mg(to3d_ctx* c);
void mg_operator_changed(to3d_ctx* c);
to3d_status mg_apply64(to3d_ctx* c, const double* r, double* z, double rnorm);
to3d_status mg_fcg_io(to3d_ctx* c, FcgIO* io);
to3d_status solve_dc_mg(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info);
to3d_status mg_capture_ready(to3d_ctx* c);
void mg_setup_launch(to3d_ctx* c, cudaStream_t s);
void mg_pcg_iter_launch(to3d_ctx* c, cudaStream_t s, int prec, int parity);
constexpr int kElementThreads = 256;   // threads per block of the element kernels
void launch_filter(to3d_ctx* c, cudaStream_t s, int mode, const double* a, const double* b,
                   double* out);
void launch_oc_begin(to3d_ctx* c, cudaStream_t s, const double* x, const double* dcf,
                     double target);
void launch_oc_passes(to3d_ctx* c, cudaStream_t s, int npass,
                      cudaGraphConditionalHandle loop = 0, int use_loop = 0);
void launch_oc_apply(to3d_ctx* c, cudaStream_t s, const double* x, double* xnew);

}  // namespace to3d
