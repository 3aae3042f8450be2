/*
 * nep.h -- C ABI of libnep: GB300-native (sm_103a) evaluation of the
 * Neuroevolution Potential (NEP) per atom and its training backward.
 *
 * The problem statement follows AI2Pot (arXiv 2607.06969), Section 2:
 *   positions + species + periodic cell  ->  E_i (Eqs. 1-2), forces (Eq. 3),
 *   virial (Eq. 4), with NEP descriptors of Eqs. 11-17;
 *   labelled configurations -> loss (Eqs. 18-21) and its parameter gradient
 *   (the paper's training operator, Section 3.2).
 *
 * Conventions for every call:
 *   - Units: eV, Angstrom, u, fs.  The virial is in eV, not divided by volume.
 *   - Every array argument is caller-owned DEVICE memory unless its name ends
 *     in _host.  The library never frees caller memory.
 *   - Per-atom arrays are structure-of-arrays: a [3][N] array holds all x,
 *     then all y, then all z.
 *   - Hot calls (nep_neighbors, nep_energy_forces_virial*, nep_param_grad*,
 *     nep_adam_step, nep_md_step, nep_md_kick, nep_md_wrap, nep_domain_*)
 *     allocate nothing and never synchronise the host; they only enqueue
 *     kernels on `stream` (a cudaStream_t, NULL = legacy default stream).
 *     Scratch memory is the caller's `work` buffer, sized by
 *     nep_workspace_bytes, or by the sizing call that the entry point names
 *     (training, FP64, slab selection).
 *   - Host-detectable argument errors return immediately with a status and a
 *     message (nep_last_error).  Device-detected conditions (neighbour list
 *     overflow, non-finite or out-of-box positions, species out of range) set
 *     flag words in nep_nlist.status; nep_check synchronises and maps them.
 *   - A model is not thread-safe; different models may be used concurrently.
 */
#ifndef NEP_H
#define NEP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NEP_OK = 0,
    NEP_ERR_ARG = 1,          /* bad argument (NULL, size, range)              */
    NEP_ERR_CUDA = 2,         /* a CUDA runtime call failed                     */
    NEP_ERR_NOMEM = 3,        /* device allocation failed (nep_create only)     */
    NEP_ERR_CAPACITY = 4,     /* neighbour list capacity exceeded; see status   */
    NEP_ERR_TIMEOUT = 5,      /* a bounded device wait gave up                  */
    NEP_ERR_STATE = 6,        /* call made in the wrong order                   */
    NEP_ERR_UNSUPPORTED = 7,  /* hyper-parameters with no compiled kernel       */
    NEP_ERR_INPUT = 8         /* device found invalid input (see nep_check)     */
} nep_status;

/* NEP hyper-parameters (Section 2.3, Table 2).
 * n_rad, n_ang : radial / angular descriptor counts, n = 0..n-1 (Eqs. 11, 16)
 * k_rad, k_ang : Chebyshev basis functions N_basis, k = 0..k-1 (Eq. 12)
 * l_max        : must be 4 (Section 2.3); l runs 1..l_max
 * has_4body    : 1 adds q4_n = tr(A_n^3), A_n = sum_j g_n (rhat rhat^T - I/3)
 * n_hidden     : hidden tanh units of the per-species network (N_neurons)
 * rc_rad/ang   : cutoffs r_max (Eqs. 13-15), rc_ang <= rc_rad
 * precision    : 0 = FP32 everywhere; 1 = MLP forward and dU/dq in FP16 on
 *                tensor cores (tcgen05, FP32 accumulation in tensor
 *                memory; descriptors FP32); 2 = same with BF16.  Precisions
 *                1 and 2 need n_hidden <= 64 (else NEP_ERR_UNSUPPORTED).
 * Descriptor dimension D = n_rad + n_ang*l_max + n_ang*has_4body, ordered
 * [q_0..q_{nR-1}, q_{n,l} (n outer, l = 1..l_max inner), q4_0..q4_{nA-1}]. */
typedef struct {
    int n_types;
    int n_rad, n_ang;
    int k_rad, k_ang;
    int l_max;
    int has_4body;
    int n_hidden;
    float rc_rad, rc_ang;
    int precision;
} nep_hparams;

typedef struct nep_model nep_model;   /* opaque, library-owned */

/* Number of parameters P.  Flat order (float):
 *   for t in types: W0[t][H][D], b0[t][H], w1[t][H], b1[t];
 *   then cR[Zi][Zj][n_rad][k_rad]; then cA[Zi][Zj][n_ang][k_ang]
 * (c indexed by the ordered species pair, Eqs. 11 and 16).
 * E_i = sum_h w1[Zi][h] tanh(sum_d W0[Zi][h][d] q_d + b0[Zi][h]) + b1[Zi].
 * Returns 0 for invalid hyper-parameters. */
size_t nep_num_params(const nep_hparams* hp);

/* Create a model from hyper-parameters and HOST parameters (P floats).
 * Allocates the model's device copy on the current device.
 * A shape with a compiled kernel set (nep_supported = 1) gets the fast path:
 * FP32, FP16 or BF16 network, every call.  Any other FP32 shape with n_rad,
 * n_ang <= 16 and k_rad, k_ang <= 16 (nep_supported = 2) gets the generic
 * path: runtime-shaped FP32 kernels that evaluate each pair term from both of
 * its atoms (about twice the fast path's pair work).  A generic model serves
 * nep_neighbors, the FP32 evaluations (nep_energy_forces_virial, _owned,
 * _noalloc), nep_md_step and the FP64 calls; nep_param_grad,
 * nep_param_grad_adjoint and nep_autotune return NEP_ERR_UNSUPPORTED (its
 * training gradient comes from nep_param_grad_fp64).  Other shapes, and
 * FP16/BF16 for shapes without a kernel set, return NEP_ERR_UNSUPPORTED. */
nep_status nep_create(const nep_hparams* hp, const float* params_host, size_t n_params,
                      nep_model** out);
nep_status nep_destroy(nep_model* m);
/* 1 if a kernel set is compiled for these hyper-parameters (the fast path),
 * 2 if only the generic FP32 path serves them, 0 if nep_create rejects them. */
int nep_supported(const nep_hparams* hp);

/* Replace the parameters from a DEVICE buffer of P floats, stream-ordered
 * (for optimiser steps that stay on the device). */
nep_status nep_set_params(nep_model* m, const float* params_dev, void* stream);

/* Copy the current parameters (P floats) into a DEVICE buffer, stream-ordered
 * (checkpoints of a training run that updates them with nep_adam_step). */
nep_status nep_get_params(const nep_model* m, float* params_dev, void* stream);

/* A batch of B periodic orthorhombic configurations with atoms concatenated.
 * pos    [3][N] float, each atom of config b inside [0, box[b][a]) for
 *        nep_neighbors (nep_energy_forces_virial accepts atoms that drifted
 *        after the list was built: pair vectors use the image stored in the
 *        list, or the minimum image when the list was built without shifts)
 * type   [N] int in [0, n_types)
 * atom_off [B+1] int CSR offsets (atom_off[0] = 0, atom_off[B] = N)
 * box    [B][3] float edge lengths
 * atom_off_host, box_host: host copies of the same values (used to plan
 * launches without a device round trip). */
typedef struct {
    int n_atoms;
    int n_cfg;
    const float* pos;
    const int* type;
    const int* atom_off;
    const float* box;
    const int* atom_off_host;
    const float* box_host;
} nep_system;

/* Verlet neighbour list, caller-owned.  For each atom i the radial list holds
 * every (j, image s) != (i, 0) with |r_j + s*L - r_i| < rc_rad + skin, decided
 * by the FP32 predicate dx = (x_j - x_i) + s_x L_x (and y, z),
 * d2 = (dx*dx + dy*dy) + dz*dz, d2 < fl32(rc*rc) (the sum over j of Eq. 3).
 * Its first cnt_ang[i] entries are exactly those with d < rc_ang + skin; the
 * remaining ones are ordered with d < rc_rad before d >= rc_rad.
 *   nbr   [cap][N] int   slot-major: nbr[s*N + i] = j
 *   shift [cap][N] int   packed image (int8 sx | sy << 8 | sz << 16); may be
 *                        NULL when every box edge >= 2*(rc_rad+skin)+1e-3,
 *                        in which case the minimum image is used
 *   rev   [cap_ang][N]   slot of i in j's angular prefix, for pair (i, s)
 *   cnt, cnt_ang [N]
 *   status [4] int: [0] overflow flag, [1] radial count needed,
 *                   [2] angular count needed, [3] bit 0: invalid input,
 *                   bit 1: a tensor-core completion wait gave up
 * nep_neighbors fills every array and the host fields skin and min_image.
 * If a count exceeds cap (cap_ang) the list is truncated, status[0] is set
 * and status[1..2] hold the capacity needed; nep_check returns
 * NEP_ERR_CAPACITY and the caller resizes and rebuilds. */
typedef struct {
    int cap, cap_ang;
    int* cnt;
    int* cnt_ang;
    int* nbr;
    int* shift;
    int* rev;
    int* status;
    float skin;     /* written by nep_neighbors */
    int min_image;  /* written by nep_neighbors */
} nep_nlist;

/* Scratch bytes needed by the hot calls for a system of N atoms, B configs,
 * and a list with capacities cap/cap_ang.  One buffer of this size serves
 * every hot call of the model. */
size_t nep_workspace_bytes(const nep_model* m, int n_atoms, int n_cfg, int cap, int cap_ang);

/* Build the cell-list Verlet list (counting sort into cells of edge
 * >= (rc + skin) / 3, a 7 x 7 x 7-cell or wider image stencil walked row by
 * row, each row cut to the cells that can meet the cutoff sphere, then a
 * reverse index).  Deterministic: list order is fixed by cell order and atom
 * index. */
nep_status nep_neighbors(nep_model* m, const nep_system* sys, float skin, nep_nlist* nl,
                         void* work, size_t work_bytes, void* stream);

/* Energies, forces and virial (Eqs. 1-4, 11-17).
 * e_atom [N] float (may be NULL), force [3][N] float,
 * e_tot [B] double, virial [B][9] double (row-major V_ab, Eq. 4).
 * Sums over atoms are FP64 in a fixed order: results are bitwise
 * reproducible run to run. */
nep_status nep_energy_forces_virial(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                    float* e_atom, float* force, double* e_tot, double* virial,
                                    void* work, size_t work_bytes, void* stream);

/* FP64 evaluation (Section 3.2: the operators run in float64 as well as
 * float32).  The same quantities as nep_energy_forces_virial with every
 * intermediate in double: positions (the FP32 inputs) are promoted, pairs
 * are kept by r < rc in double, and per-atom E and W_i = -sum_j
 * dE_i/dr_ij (x) r_ij are summed in FP64 in a fixed order.  The list is an
 * nep_neighbors list (cnt, nbr, shift or minimum image); pairs that the FP32
 * list predicate left out are not seen.
 *   params : [P] double DEVICE parameters in the layout of nep_create, or
 *            NULL for the model's FP32 parameters promoted to double
 *   e_atom [N] double (may be NULL), force [3][N] double,
 *   e_tot [B] double, virial [B][9] double (row-major V_ab, Eq. 4)
 *   work   : >= nep_workspace_bytes_fp64(m, N, B) bytes, 256-byte aligned
 * One thread per atom; every pair term is evaluated by both of its atoms, so
 * the call is deterministic and allocation-free.  Needs n_rad, n_ang <= 16 and
 * k_rad, k_ang <= 16 (else NEP_ERR_UNSUPPORTED); any precision setting. */
size_t nep_workspace_bytes_fp64(const nep_model* m, int n_atoms, int n_cfg);
nep_status nep_energy_forces_virial_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                         const double* params, double* e_atom, double* force,
                                         double* e_tot, double* virial, void* work, size_t work_bytes,
                                         void* stream);

/* FP64 loss and gradient (the training operator of Sections 3.2-3.3 in
 * float64): the quantities of nep_param_grad / nep_param_grad_adjoint with
 * every intermediate in double, on the FP64 evaluation above.
 *   params : [P] double DEVICE parameters, or NULL for the model's FP32
 *            parameters promoted to double
 *   e_lbl [B] double, f_lbl [3][N] double, v_lbl [B][9] double,
 *   w_host[3] = (wE, wF, wV), loss_mode 0 or 1 (as nep_param_grad)
 *   grad [P] double (overwritten), loss [1] double (may be NULL)
 *   work   : >= nep_train_workspace_bytes_fp64(m, N, B) bytes, 256-byte aligned
 * Per atom: descriptors, network, the tangent of q along
 * dr_ij = -(lam_j - lam_i) - mu r_ij, the network's second-order terms and
 * the per-pair angular coefficients, recomputed (nothing cached across
 * calls); the parameter sums run per 1,024-atom chunk and then over chunks,
 * in a fixed order.  Needs, besides the FP64 evaluation's limits,
 * n_types * n_ang * k_ang <= 256 (else NEP_ERR_UNSUPPORTED). */
size_t nep_train_workspace_bytes_fp64(const nep_model* m, int n_atoms, int n_cfg);
nep_status nep_param_grad_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl, const double* params,
                               const double* e_lbl, const double* f_lbl, const double* v_lbl,
                               const float* w_host, int loss_mode, double* grad, double* loss, void* work,
                               size_t work_bytes, void* stream);
/* The gradient of Phi = sum_b a_e[b] E_b + sum_i lam[:,i] . F_i
 * + sum_b mu[b] : V_b at fixed adjoints, in FP64: a_e [B], lam [3][N],
 * mu [B][9] double; grad [P] double.  The vector-Jacobian product of an
 * FP64 autograd backward. */
nep_status nep_param_grad_adjoint_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                       const double* params, const double* a_e, const double* lam,
                                       const double* mu, double* grad, void* work, size_t work_bytes,
                                       void* stream);

/* nep_energy_forces_virial with the per-configuration sums restricted to
 * the atoms [0, n_owned): forces (and e_atom) are computed for every atom,
 * e_tot and virial sum only the first n_owned.  The evaluation of one rank's
 * local system in a spatial decomposition, whose owned atoms come first and
 * whose ghost atoms follow (nep_domain_select). */
nep_status nep_energy_forces_virial_owned(nep_model* m, const nep_system* sys, const nep_nlist* nl, int n_owned,
                                          float* e_atom, float* force, double* e_tot, double* virial, void* work,
                                          size_t work_bytes, void* stream);

/* The velocity-Verlet pieces of nep_md_step, for callers that evaluate the
 * forces themselves (a spatial decomposition): per atom v += half_dt F/m
 * (masses_host[n_types] in u, F in eV/A, v in A/fs), then, if drift_dt > 0,
 * x += drift_dt v.  nep_md_wrap wraps every atom into its configuration's
 * box, as nep_md_step does at a rebuild.  sys->pos is written.
 * NEP_ERR_ARG: masses_host NULL or a mass <= 0, vel or force NULL, half_dt
 * not finite, drift_dt negative or not finite. */
nep_status nep_md_kick(nep_model* m, const nep_system* sys, float* vel, const float* force, const float* masses_host,
                       float half_dt, float drift_dt, void* stream);
nep_status nep_md_wrap(nep_model* m, const nep_system* sys, void* stream);

/* Spatial decomposition of one periodic configuration into slabs along x,
 * for a multi-GPU run of one large system.  A rank owns the atoms with
 * x in [x_lo, x_hi) and evaluates them with the ghost atoms within `halo` of
 * its slab (for each ghost, the image in [x_lo - halo, x_hi + halo)).  With
 * halo >= 2 (rc_rad + skin), the owned atoms' energies, forces and per-atom
 * virials equal those of the whole-system evaluation; the ranks then combine
 * their owned rows (one all-reduce of the forces, energies and virials).
 *
 * nep_domain_select: pos [3][N] device (x wrapped into [0, box_host[0])),
 *   idx [cap], img [cap] device outputs: owned atoms, then ghosts, each in
 *   atom order; img = the ghost's image in units of box x (0 for owned);
 *   counts [2] device: owned, owned + ghosts (entries beyond cap are not
 *   written: the caller compares counts[1] with cap and selects again).
 *   Needs 0 <= x_lo < x_hi <= box x and slab + 2 halo <= box x.  work:
 *   nep_domain_workspace_bytes(N) bytes.  Deterministic.
 * nep_domain_gather: the n_local selected atoms into the local frame,
 *   pos_local [3][n_local] = (x + img box_x - x_origin, y, z) and
 *   type_local [n_local].
 * nep_domain_scatter: dst[c][idx[l]] = src[c][l] for the owned rows
 *   l < n_owned, c < ncomp (src [ncomp][n_local], dst [ncomp][N]); the
 *   other entries of dst are left as they are. */
size_t nep_domain_workspace_bytes(int n_atoms);
nep_status nep_domain_select(const float* pos, int n_atoms, const float* box_host, float x_lo, float x_hi,
                             float halo, int* idx, int* img, int cap, int* counts, void* work, size_t work_bytes,
                             void* stream);
nep_status nep_domain_gather(const float* pos, const int* type, int n_atoms, const int* idx, const int* img,
                             int n_local, const float* box_host, float x_origin, float* pos_local, int* type_local,
                             void* stream);
nep_status nep_domain_scatter(const float* src, int n_local, int ncomp, const int* idx, int n_owned, float* dst,
                              int n_atoms, void* stream);

/* Point-to-point halo of a slab decomposition (Section 3.5's one domain per
 * device, with ghosts moved between neighbouring ranks only).  Each rank keeps
 * just its own atoms; every step it sends the positions of its atoms within
 * the halo of each slab face to the neighbouring rank across that face and
 * receives that rank's ghosts; at a rebuild, atoms that left the slab move to
 * the neighbour with their velocities.
 * nep_domain_band: idx [cap] device output: the atoms with x in [x_lo, x_hi)
 *   (either bound may be infinite), in atom order; counts [2] device: the
 *   count, twice (entries beyond cap are not written).  pos [3][N] device;
 *   work: nep_domain_workspace_bytes(N).  NEP_ERR_ARG unless x_lo < x_hi.
 * nep_domain_take: dst [ncomp][n] = src [ncomp][n_src] at columns idx[0..n),
 *   32-bit words copied bit for bit (positions, velocities, species, ids).
 * nep_domain_place: dst[c * dst_stride + dst_offset + l] = src[c * n + l]
 *   (src [ncomp][n], 32-bit words).  When box_x > 0, component 0 is an x
 *   coordinate: it is moved by the multiple of box_x that brings it nearest
 *   x_center (x - box_x rint((x - x_center)/box_x)) and taken relative to
 *   x_origin; every other word, and every word when box_x <= 0, is copied bit
 *   for bit.  NEP_ERR_ARG unless 0 <= dst_offset and dst_offset + n <=
 *   dst_stride, or if box_x, x_center or x_origin is not finite. */
nep_status nep_domain_band(const float* pos, int n_atoms, float x_lo, float x_hi, int* idx, int cap, int* counts,
                           void* work, size_t work_bytes, void* stream);
nep_status nep_domain_take(const void* src, int n_src, int ncomp, const int* idx, int n, void* dst, void* stream);
nep_status nep_domain_place(const void* src, int n, int ncomp, float box_x, float x_center, float x_origin,
                            void* dst, int dst_stride, int dst_offset, void* stream);

/* nep_energy_forces_virial without a caller workspace.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory at all -- for example a force plugin inside a host MD code
 * whose engine reserves the device memory and hands plugins no scratch
 * buffers, or a real-time loop that forbids allocator calls after start-up
 * because cudaMalloc/cudaFree may synchronise the whole device.
 *
 * Scratch comes from one file-scope device array of NEP_NOALLOC_SCRATCH_BYTES
 * (32 MiB) that every GPU loading the library holds until the process exits.
 * The call allocates nothing: no cudaMalloc, no cudaFree, no allocating
 * library routine.  Inputs, the neighbour list and the outputs are the
 * caller's, exactly as for nep_energy_forces_virial, and the results are the
 * same.  A system whose scratch (nep_workspace_bytes) exceeds the array is
 * rejected with NEP_ERR_ARG and a message giving both sizes.
 *
 * The first call on a device looks up the array's device address for that
 * device (cudaGetSymbolAddress, once per device, with the caller's device
 * current); make that first call before any stream capture.  The address
 * is cached for the life of the process: it belongs to the device's primary
 * context, so after cudaDeviceReset (or any other teardown of that context)
 * it is stale and this entry point must not be called again in that
 * process.  Every call
 * shares the one array and leaves its contents behind; the computation
 * writes every scratch word it later reads, so nothing needs clearing
 * between calls.  Calls whose GPU work overlaps (different streams, or
 * several host threads) race on the array and must be serialised by the
 * caller. */
#define NEP_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
nep_status nep_energy_forces_virial_noalloc(nep_model* m, const nep_system* sys,
                                            const nep_nlist* nl, float* e_atom, float* force,
                                            double* e_tot, double* virial, void* stream);

/* Scratch bytes of nep_param_grad / nep_param_grad_adjoint (the evaluation
 * scratch plus the training intermediates: descriptors, their tangents,
 * per-pair adjoint coefficients and per-chunk gradient partials). */
size_t nep_train_workspace_bytes(const nep_model* m, int n_atoms, int n_cfg, int cap, int cap_ang);

/* Loss and its gradient with respect to all P parameters (Eqs. 18-21).
 * e_lbl [B] double, f_lbl [3][N] float, v_lbl [B][9] double,
 * w_host[3] = (wE, wF, wV).
 * loss_mode 0: L = 1/B sum_b [wE (dE_b/N_b)^2 + wF/(3N_b) sum_i |dF_i|^2
 *                             + wV/9 sum_ab (dV_b,ab/N_b)^2]
 * loss_mode 1: Eqs. 19-21 per configuration, averaged over the batch:
 *              1/B sum_b [wE dE_b^2/N_b + wF/(3N_b) sum |dF|^2 + wV/(9N_b) sum dV^2]
 * A configuration with no atoms adds no term (its per-atom normalisation is
 * undefined) but counts in B.
 * grad [P] float (overwritten), loss [1] double (may be NULL).
 * work: nep_train_workspace_bytes bytes.  The gradient is that of the FP32
 * forward; sums over atoms and chunks are fixed-order (FP64 across chunks),
 * so results are bitwise reproducible.  Per-pair derivatives are
 * recomputed; nothing is cached across calls. */
nep_status nep_param_grad(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                          const double* e_lbl, const float* f_lbl, const double* v_lbl,
                          const float* w_host, int loss_mode, float* grad, double* loss,
                          void* work, size_t work_bytes, void* stream);

/* Gradient of Phi = sum_b a_e[b] E_b + sum_i lam[:,i] . F_i + sum_b mu[b] : V_b
 * with the adjoints held fixed (the vector-Jacobian product used by an
 * autograd backward).  a_e [B] double, lam [3][N] float, mu [B][9] double.
 * grad [P] float (overwritten).  work: nep_train_workspace_bytes bytes. */
nep_status nep_param_grad_adjoint(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                  const double* a_e, const float* lam, const double* mu,
                                  float* grad, void* work, size_t work_bytes, void* stream);

/* One Adam step on the model's own parameters (the optimiser of the
 * training protocol, Section 3.3.1; Kingma and Ba's update with PyTorch's
 * arrangement of the bias corrections):
 *   m = beta1 m + (1 - beta1) g,   v = beta2 v + (1 - beta2) g^2,
 *   theta -= lr / (1 - beta1^t) * m / (sqrt(v) / sqrt(1 - beta2^t) + eps)
 * grad [P] float (e.g. from nep_param_grad), m1 [P] and m2 [P] float are the
 * caller's moment buffers (zero before step t = 1), t >= 1 the step number.
 * No weight decay.  A hot call: one kernel on `stream`, no allocation.
 * NEP_ERR_ARG: a NULL buffer, t < 1, lr negative or not finite, beta1 or
 * beta2 outside [0, 1), eps <= 0 or not finite. */
nep_status nep_adam_step(nep_model* m, const float* grad, float* m1, float* m2, int t, float lr,
                         float beta1, float beta2, float eps, void* stream);

/* One velocity-Verlet step (dt in fs, masses_host[n_types] in u):
 *   v += dt/2 F/m; x += dt v; [wrap + rebuild list if rebuild != 0];
 *   F = force(x); v += dt/2 F/m.
 * pos is updated in place (sys->pos is treated as writable), vel [3][N],
 * force [3][N] must hold the forces of the current positions on entry
 * (call nep_energy_forces_virial once before the first step).
 * e_tot/virial receive the new step's values.
 * NEP_ERR_ARG: the system or list checks of nep_neighbors, masses_host NULL
 * or a mass <= 0, vel or force NULL, dt <= 0 or not finite, a workspace
 * smaller than nep_workspace_bytes. */
nep_status nep_md_step(nep_model* m, const nep_system* sys, nep_nlist* nl, float* vel,
                       float* force, double* e_tot, double* virial, const float* masses_host,
                       float dt, float skin, int rebuild, void* work, size_t work_bytes,
                       void* stream);

/* Autotuner: on this system and list, times the launch choices of the three
 * pair kernels, `reps` timed launches each after one untimed launch:
 *   the radial kernel at 64, 128 and 256 threads per block;
 *   every compiled register-budget variant of the angular kernel (the
 *   register-heavy one: 2, 3 or 4 resident blocks of 128 threads per SM);
 *   the finish kernel at 64, 128 and 256 threads per block.
 * The fastest of each is stored in the model for the system's size class
 * (log2 of the mean atom count per configuration); later hot calls on
 * systems of that class use them.  Small systems gain from small blocks (more
 * blocks cover more SMs); large ones do not care.  Not a hot call: it
 * synchronises `stream` and overwrites the workspace's scratch.
 * chosen[3] (may be NULL) receives the angular variant index (0, 1, 2 = 2, 3,
 * 4 blocks per SM), the radial and the finish block size.  Untuned classes
 * use variant 0, 256 (radial) and 128 (finish). */
nep_status nep_autotune(nep_model* m, const nep_system* sys, const nep_nlist* nl, void* work,
                        size_t work_bytes, void* stream, int reps, int* chosen);

/* Pin the angular kernel variant (0, 1, 2 = 2, 3, 4 resident blocks per SM;
 * -1 = back to the default) for one size class (0..31, as in nep_autotune)
 * or for all of them (size_class = -1).  Host only, no device work. */
nep_status nep_set_variant(nep_model* m, int size_class, int variant);

/* Pin every launch choice of nep_autotune for one size class or all of them
 * (size_class = -1): the angular variant (-1 = default) and the radial and
 * finish block sizes (64, 128, 256, or 0 = default).  Host only.
 * NEP_ERR_ARG for any other value. */
nep_status nep_set_launch(nep_model* m, int size_class, int variant, int radial_block, int finish_block);

/* Profiling hook: the next nep_energy_forces_virial / nep_md_step call of
 * this model records events[0] before the radial kernel (radial sums,
 * angular pair compaction), events[1] after it, events[2] after the angular
 * kernel (angular descriptors, network, angular pair forces) and events[3]
 * after the kernel that completes the forces, on the call's stream (events
 * are caller-created cudaEvent_t, n = 4; n = 0 clears).  One-shot: the
 * events are forgotten after that call.  The records are ordinary stream work
 * and can be captured into a CUDA graph. */
nep_status nep_set_timing_events(nep_model* m, void* const* events, int n);

/* Measurement helper, not part of the NEP path: the FP32 FMA throughput of
 * the device, from a kernel of independent FMA chains on every SM, timed
 * with CUDA events on `stream` (synchronises).  *tflops receives 2 flops per
 * FMA per second / 1e12. */
nep_status nep_fp32_peak(void* stream, double* tflops);

/* Self-test of the bounded tensor-core completion wait, not part of the NEP
 * path: one CTA allocates tensor memory, waits on an mbarrier that nothing
 * arrives at with a short poll limit, records the timeout in a device flag,
 * frees its columns and returns; the host reads the flag.  Returns
 * NEP_ERR_TIMEOUT when the wait ran out as designed (the CUDA context stays
 * usable), NEP_OK if the wait completed, or a CUDA error.  Synchronises. */
nep_status nep_selftest_wait_timeout(void* stream);

/* Synchronise `stream` and map the list's device flags to a status:
 * NEP_ERR_CAPACITY (status[0]), NEP_ERR_TIMEOUT (status[3] bit 1),
 * NEP_ERR_INPUT (status[3] bit 0) or NEP_OK.
 * nl may be NULL (then only the stream is synchronised). */
nep_status nep_check(const nep_nlist* nl, void* stream);

/* Thread-local message of the last failed call ("" if none). */
const char* nep_last_error(void);

/* Library version string. */
const char* nep_version(void);

#ifdef __cplusplus
}
#endif
#endif /* NEP_H */
