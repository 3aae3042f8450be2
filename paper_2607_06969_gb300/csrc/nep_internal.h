// Internal declarations shared by the translation units of libnep.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "nep.h"

#if defined(__CUDACC__)
#define NEP_HD __host__ __device__ __forceinline__
#else
#define NEP_HD inline
#endif

namespace nep {

// largest hidden width of the FP16/BF16 tensor-core network
constexpr int kTcMaxHidden = 64;
constexpr int kMaxTypes = 4;
constexpr int kLM = 24;          // real solid harmonics for l = 1..4: 3+5+7+9
constexpr int kChunk = 1024;     // atoms per reduction chunk (one CTA)
constexpr int kBlock = 128;      // threads per block of the per-atom kernels
constexpr int kVariants = 3;              // angular kernel register budgets: 2, 3, 4 blocks per SM
constexpr int kDefaultAngularVariant = 0; // 2 blocks per SM, S_nlm in tensor memory
constexpr int kSizeBins = 32;             // tuning table: log2 of mean atoms per configuration
constexpr int kBlockChoices[3] = {64, 128, 256};   // block sizes the tuner tries for radial / finish
constexpr int kRowStride = 64;            // list build: bytes of per-atom stencil row starts

// Stencil/cell plan of one configuration for the neighbour build.
struct CellPlan {
    int nc[3];     // cells per edge
    int half[3];   // stencil half-width per edge
    int base;      // first global cell id
    int pad;
};

// Everything the per-atom kernels read or write.  All pointers are device
// pointers (or host pointers when the same code runs in a host emulation).
struct EvalArgs {
    int N, B, T, H;
    int cap, cap_ang;
    int min_image;
    float rc_rad, rc_ang;          // physics cutoffs
    const float4* pos4;            // [N] x, y, z, type bits
    const int* cfg;                // [N] configuration of each atom
    const float* box;              // [B][3]
    const int* cnt;                // [N]
    const int* cnt_ang;            // [N]
    const int* nbr;                // [cap][N]
    const int* shift;              // [cap][N] or null
    const int* rev;                // [cap_ang][N]
    const float* params;           // [P] flat model parameters
    // per-atom scratch
    float* e_atom;                 // [N]
    float* fb;                     // [T*KR][N]       species-resolved radial basis sums
    float* S;                      // [NA*24][N]      S_nlm (mixed precision and training only)
    float* Pr;                     // [N][T][KR]      sum_n dE/dq_n cR[Zi][t][n][k]
    float4* comp;                  // [cap_ang][N]    compacted angular pairs
    int* cnt_comp;                 // [N]
    float4* compr;                 // [cap][N]        compacted radial pairs (r_ij, j|tj), training only
    int* cnt_compr;                // [N]
    unsigned long long* amask;     // [N] angular-prefix slots below 64 that lie inside rc_ang (with compr)
    int* rin;                      // [cap][N]        list entries after the angular prefix that lie
    int* rin_sh;                   // [cap][N]        inside rc_rad (j; image shift or null), in
    int* cnt_rin;                  // [N]             list order, written by the radial kernel
    float4* fin;                   // [cap_ang][N]    incoming angular pair forces
    float* fpart;                  // [3][N]
    float* wat;                    // [9][N]          per-atom virial
    int* status;                   // [4] flags (may be null)
    // network precision: 0 FP32 (CUDA cores), 1 FP16, 2 BF16 (tensor cores)
    int q16_kind;
    // training outputs of the angular kernel (null when not training)
    float* q_out;                  // [D][N]          descriptors
    float* p_out;                  // [D][N]          dE/dq
    float* fb_out;                 // [T*KR][N]       species-resolved radial basis sums
};

// Inputs and scratch of the training backward (see nep_train.cuh).
struct TrainArgs {
    EvalArgs e;
    const float4* lam4;            // [N]  force adjoint lambda_i = dL/dF_i
    const float* aE;               // [B]  energy adjoint dL/dE_b
    const float* mu;               // [B][9] virial adjoint dL/dV_b
    float* dq;                     // [D][N]   tangent of q along dr
    float* dS;                     // [NA*24][N]
    float* df;                     // [T*KR][N]
    float* coef;                   // [3H][N]  alpha, beta, gamma of the network gradient
    float* rho;                    // [D][N]   a dE/dq + d(dE/dq . dq)/dq
    float* xz;                     // [3*NA][cap_ang][N] per angular pair: X_n from P, Z_n, X_n from R
    float* bins;                   // [T*NA*KA][N] per-atom angular c-gradient
    float* gpart;                  // [chunks][P] per-chunk gradient partials
    float* grad;                   // [P] output
};

// Outputs of the force-completion kernel.
struct FinishArgs {
    const int* atom_off;           // [B+1]
    const int* chunk_start;        // [B+1] reduction chunks per configuration
    double* partial;               // [chunks][10] FP64 E and virial per chunk
    float* force;                  // [3][N]
    float* e_out;                  // [N] or null
    int n_owned;                   // atoms [0, n_owned) enter the E and virial sums
};

// Offsets of the parameter blocks in the flat vector.
struct ParamLayout {
    int D, P;
    int mlp_stride;   // per type: H*D + 2H + 1
    int off_cR, off_cA;
};

NEP_HD ParamLayout param_layout(int T, int NR, int NA, int KR, int KA, int H4, int H) {
    ParamLayout L;
    L.D = NR + NA * 4 + (H4 ? NA : 0);
    L.mlp_stride = H * L.D + 2 * H + 1;
    L.off_cR = T * L.mlp_stride;
    L.off_cA = L.off_cR + T * T * NR * KR;
    L.P = L.off_cA + T * T * NA * KA;
    return L;
}

// A compiled hyper-parameter instance: launchers for its kernels.
struct KernelSet {
    int n_rad, n_ang, k_rad, k_ang, has_4body, n_types;
    size_t (*smem_bytes)(int H);
    cudaError_t (*init)(int H);   // set kernel attributes (dynamic shared memory)
    // block: threads per block of the radial / finish kernel, one of
    // kBlockChoices, or 0 for the kernel's default
    cudaError_t (*radial)(const EvalArgs&, cudaStream_t, int block);
    cudaError_t (*angular)(const EvalArgs&, cudaStream_t, int variant);   // FP32 or tensor-core network
    cudaError_t (*finish)(const EvalArgs&, const FinishArgs&, int max_chunks, cudaStream_t, int block);
    cudaError_t (*train_init)(int H);
    cudaError_t (*train)(const TrainArgs&, cudaStream_t);   // tangent ... gradient
    int (*grad_chunks)(int N);
};

const KernelSet* find_kernel_set(int n_rad, int n_ang, int k_rad, int k_ang, int has_4body,
                                 int n_types);

// runtime kernels (nep_runtime.cu)
cudaError_t launch_pack(const float* pos, const int* type, const int* atom_off, int N, int B,
                        int T, float4* pos4, int* cfg, int* status, cudaStream_t st);
cudaError_t launch_chunk_plan(const int* atom_off, int B, int* chunk_start, cudaStream_t st);
// FP64 sums of E_i and the per-atom virials per reduction chunk
cudaError_t launch_chunk_reduce(const EvalArgs& a, const FinishArgs& f, int max_chunks, cudaStream_t st);
cudaError_t launch_final_reduce(int B, const int* chunk_start, const double* partial,
                                double* e_tot, double* virial, cudaStream_t st);

struct NbrWork {
    CellPlan* plan;        // [B]
    int* cell_of;          // [N]
    int* rank;             // [N]
    int* cell_cnt;         // [Cmax]
    int* cell_start;       // [Cmax+1]
    int* cell_atoms;       // [N]
    float4* cell_pos;      // [N] positions in cell order, atom index bits in w
    int* scan_tmp;         // [ceil(Cmax/2048)+1]
    int2* shell;           // [cap][N] scratch for the list entries beyond rc_rad
    unsigned char* row_start;   // [N][32] where each stencil row's angular entries start
    unsigned char* slot_row;    // [cap_ang][N] stencil row of each angular entry
    int cmax;
};
size_t nbr_cell_capacity(int N, int B);
cudaError_t launch_neighbors(const float* pos, const float4* pos4, const int* atom_off, const float* box,
                             const int* cfg, int N, int B, float rc_list, float rc_list_ang, float rc_phys,
                             int min_image, nep_nlist* nl, const NbrWork& w, cudaStream_t st);

// FP64 evaluation and training gradient (nep_fp64.cu): runtime
// hyper-parameters, every quantity in double.  Bounds of the per-thread
// arrays:
constexpr int kF64MaxN = 16;      // n_rad, n_ang
constexpr int kF64MaxK = 16;      // k_rad, k_ang
constexpr int kF64MaxBins = 256;  // n_types * n_ang * k_ang (training gradient)
// The generic FP32 evaluation (any hyper-parameters within the FP64 path's
// bounds): the evaluation fields of F64Args, in float.  The FP64 path's
// evaluation kernels are templates over the two.
struct F32Args {
    int N, B, T, NR, NA, KR, KA, H, H4, D;
    ParamLayout L;
    float rc_rad, rc_ang;
    const float* pos;              // [3][N]
    const int* type;               // [N]
    const int* cfg;                // [N]
    const float* box;              // [B][3]
    const int* cnt;                // [N]
    const int* nbr;                // [cap][N]
    const int* shift;              // [cap][N] packed images, or null (minimum image)
    const float* prm;              // [P]
    float* e;                      // [N]     E_i
    float* p;                      // [NR][N] dE_i/dq_n, radial n
    float* R;                      // [NA*24][N] dE_i/dS_nlm
    float* w;                      // [9][N]  per-atom virial
    float* force;                  // [3][N]
    const int* atom_off;           // [B+1]
    const int* chunk_start;        // [B+1]
    double* partial;               // [chunks][10]
    int n_owned;                   // atoms [0, n_owned) enter the E and virial sums
};
cudaError_t launch_efv_generic(const F32Args& a, int max_chunks, double* e_tot, double* virial,
                               cudaStream_t st);

struct F64Args {
    int N, B, T, NR, NA, KR, KA, H, H4, D;
    ParamLayout L;
    double rc_rad, rc_ang;
    const float* pos;              // [3][N]
    const int* type;               // [N]
    const int* cfg;                // [N]
    const float* box;              // [B][3]
    const int* cnt;                // [N]
    const int* nbr;                // [cap][N]
    const int* shift;              // [cap][N] packed images, or null (minimum image)
    const double* prm;             // [P]
    double* e;                     // [N]     E_i
    double* p;                     // [NR][N] dE_i/dq_n, radial n
    double* R;                     // [NA*24][N] dE_i/dS_nlm
    double* w;                     // [9][N]  per-atom virial
    double* force;                 // [3][N]
    const int* atom_off;           // [B+1]
    const int* chunk_start;        // [B+1]
    double* partial;               // [chunks][10]
    int n_owned;                   // atoms [0, n_owned) enter the E and virial sums
    // training gradient
    const double* lam;             // [3][N] dL/dF
    const double* aE;              // [B]    dL/dE
    const double* mu;              // [B][9] dL/dV
    double* st;                    // [fields][N] per-atom gradient factors
    double* gpart;                 // [gradient chunks][P]
    double* grad;                  // [P]
};
cudaError_t launch_promote(const float* src, double* dst, int n, cudaStream_t st);
int fp64_lanes_per_atom(int N);
int fp64_grad_fields(const F64Args& a);
int fp64_grad_chunks(int N);
cudaError_t launch_efv_fp64(const F64Args& a, int max_chunks, double* e_tot, double* virial,
                            cudaStream_t st);
// loss (Eqs. 18-21, modes as nep_param_grad) and its adjoints from the FP64
// forces, energies and virials
cudaError_t launch_loss_fp64(const F64Args& a, int max_chunks, const double* e_tot, const double* vir,
                             const double* e_lbl, const double* f_lbl, const double* v_lbl, const float* w,
                             int mode, double* lam, double* aE, double* mu, double* loss, cudaStream_t st);
cudaError_t launch_grad_fp64(const F64Args& a, cudaStream_t st);

// slab decomposition along x (nep_domain.cu)
size_t domain_scratch_bytes(int N);
cudaError_t launch_domain_select(const float* pos, int N, float Lx, float lo, float hi, float halo, int* idx,
                                 int* img, int cap, int* counts, void* scratch, cudaStream_t st);
cudaError_t launch_domain_gather(const float* pos, const int* type, int N, const int* idx, const int* img,
                                 int n_local, float Lx, float x_origin, float* pos_local, int* type_local,
                                 cudaStream_t st);
cudaError_t launch_domain_scatter(const float* src, int n_local, int ncomp, const int* idx, int n_owned,
                                  float* dst, int N, cudaStream_t st);
cudaError_t launch_domain_take(const void* src, int n_src, int ncomp, const int* idx, int n, void* dst,
                               cudaStream_t st);
cudaError_t launch_domain_place(const void* src, int n, int ncomp, float box_x, float x_center, float x_origin,
                                void* dst, int stride, int offset, cudaStream_t st);

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float beta1, float beta2,
                        float eps, float c1, float c2, cudaStream_t st);
cudaError_t fp32_peak(cudaStream_t st, double* tflops);
cudaError_t wait_selftest(cudaStream_t st, int* outcome);
cudaError_t launch_kick(float* vel, const float* force, const int* type, const float* inv_mass,
                        int N, float half_dt, float* pos, float dt, cudaStream_t st);
cudaError_t launch_wrap(float* pos, const int* cfg, const float* box, int N, cudaStream_t st);
cudaError_t launch_wrap_segments(float* pos, const int* atom_off, int B, const float* box, int N, cudaStream_t st);
cudaError_t launch_loss(int N, int B, const int* atom_off, const int* chunk_start, int max_chunks,
                        const float* force, const float* f_lbl, const double* e_tot,
                        const double* vir, const double* e_lbl, const double* v_lbl,
                        const float* w, int mode, float4* lam4, float* aE, float* mu,
                        double* partial, double* loss, cudaStream_t st);
cudaError_t launch_pack_adjoint(int N, int B, const float* lam, const double* a_e, const double* mu_in,
                                float4* lam4, float* aE, float* mu, cudaStream_t st);

}  // namespace nep
