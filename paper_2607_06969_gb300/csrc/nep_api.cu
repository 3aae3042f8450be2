// C ABI of libnep (declared in include/nep.h): argument checks, workspace
// carving and kernel dispatch.  No allocation and no host synchronisation
// happens in the hot calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <mutex>

#include "nep_internal.h"

struct nep_model {
    nep_hparams hp;
    const nep::KernelSet* ks;   // compiled fast path; null: the generic FP32 path (runtime shapes)
    nep::ParamLayout lay;
    float* params;   // device [P]
    int device;
    cudaEvent_t timing[4];
    int n_timing;
    // autotuned launch choices per size class (-1 / 0: default)
    int tune_angular[nep::kSizeBins];   // angular kernel variant per size class, -1 = default
    int tune_radial[nep::kSizeBins];    // radial kernel block size per size class, 0 = default
    int tune_finish[nep::kSizeBins];    // finish kernel block size per size class, 0 = default
};

namespace {

thread_local std::string g_err;

nep_status fail(nep_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

nep_status cuda_fail(cudaError_t e, const char* where) {
    return fail(NEP_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NEP_CUDA(call, where)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool hp_valid(const nep_hparams* hp) {
    return hp && hp->n_types >= 1 && hp->n_types <= nep::kMaxTypes && hp->n_rad >= 1 &&
           hp->n_ang >= 1 && hp->k_rad >= 1 && hp->k_ang >= 1 && hp->l_max == 4 &&
           (hp->has_4body == 0 || hp->has_4body == 1) && hp->n_hidden >= 1 &&
           hp->n_hidden <= 1024 && hp->rc_rad > 0.0f && hp->rc_ang > 0.0f &&
           hp->rc_ang <= hp->rc_rad && hp->precision >= 0 && hp->precision <= 2 &&
           std::isfinite(hp->rc_rad) && std::isfinite(hp->rc_ang);
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the scratch arrays inside the caller's workspace.
struct WsLayout {
    size_t pos4, cfg, e_atom, fb, S, Pr, comp, cnt_comp, fin, fpart, wat, chunk_start, partial;
    size_t rin, rin_sh, cnt_rin;
    size_t amask;
    size_t gen_p, gen_R, gen_w;   // generic FP32 path: dE/dq (radial), dE/dS, per-atom virial
    size_t plan, cell_of, rank, cell_cnt, cell_start, cell_atoms, cell_pos, scan_tmp, shell, row_start, slot_row;
    size_t total;
    int max_chunks, cmax;
};

WsLayout ws_layout(const nep_model* m, int N, int B, int cap, int cap_ang) {
    WsLayout w;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t n = (size_t)N;
    const int NA = m->hp.n_ang, T = m->hp.n_types, KR = m->hp.k_rad;
    w.pos4 = take(16 * n);
    w.cfg = take(4 * n);
    w.e_atom = take(4 * n);
    w.fb = take(4 * n * T * KR);
    // S and the angular dE/dq leave the SM only in mixed precision and training
    w.S = take(4 * n * NA * nep::kLM);
    w.Pr = take(4 * n * T * KR);
    w.comp = take(16 * n * cap_ang);
    w.cnt_comp = take(4 * n);
    w.fin = take(16 * n * cap_ang);
    w.rin = take(4 * n * cap);
    w.rin_sh = take(4 * n * cap);
    w.cnt_rin = take(4 * n);
    w.amask = take(8 * n);
    if (!m->ks) {
        w.gen_p = take(4 * n * m->hp.n_rad);
        w.gen_R = take(4 * n * NA * nep::kLM);
        w.gen_w = take(36 * n);
    } else {
        w.gen_p = w.gen_R = w.gen_w = 0;
    }
    w.fpart = take(12 * n);
    w.wat = take(36 * n);
    w.chunk_start = take(4 * ((size_t)B + 1));
    w.max_chunks = (int)((n + nep::kChunk - 1) / nep::kChunk) + B;
    w.partial = take(80 * (size_t)w.max_chunks);
    w.cmax = (int)nep::nbr_cell_capacity(N, B);
    w.plan = take(sizeof(nep::CellPlan) * (size_t)B);
    w.cell_of = take(4 * n);
    w.rank = take(4 * n);
    w.cell_cnt = take(4 * ((size_t)w.cmax + 1));
    w.cell_start = take(4 * ((size_t)w.cmax + 1));
    w.cell_atoms = take(4 * n);
    w.cell_pos = take(16 * n);
    const size_t ntiles = ((size_t)w.cmax + 1 + 2047) / 2048;
    w.scan_tmp = take(4 * (ntiles + 1));
    w.shell = take(8 * n * (size_t)cap);
    w.row_start = take((size_t)nep::kRowStride * n);
    w.slot_row = take(n * (size_t)cap_ang);
    w.total = o;
    return w;
}

// Training scratch placed after the evaluation scratch.
struct TrainLayout {
    WsLayout w;
    size_t q, p, compr, cnt_compr, lam4, aE, mu, partialF, etot, vir, force, dq, dS, df, coef, rho, xz,
        bins, gpart, loss;
    size_t total;
};

TrainLayout train_layout(const nep_model* m, int N, int B, int cap, int cap_ang) {
    TrainLayout t;
    t.w = ws_layout(m, N, B, cap, cap_ang);
    size_t o = t.w.total;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t n = (size_t)N;
    const int D = m->lay.D, NA = m->hp.n_ang, T = m->hp.n_types, KR = m->hp.k_rad, KA = m->hp.k_ang;
    const int H = m->hp.n_hidden;
    t.q = take(4 * n * D);
    t.p = take(4 * n * D);
    t.compr = take(16 * n * (size_t)cap);
    t.cnt_compr = take(4 * n);
    t.lam4 = take(16 * n);
    t.aE = take(4 * (size_t)B);
    t.mu = take(36 * (size_t)B);
    t.partialF = take(8 * (size_t)t.w.max_chunks);
    t.etot = take(8 * (size_t)B);
    t.vir = take(72 * (size_t)B);
    t.force = take(12 * n);
    t.dq = take(4 * n * D);
    t.dS = take(4 * n * NA * nep::kLM);
    t.df = take(4 * n * T * KR);
    t.coef = take(4 * n * 3 * H);
    t.rho = take(4 * n * D);
    t.xz = take(4 * n * 3 * NA * (size_t)cap_ang);
    t.bins = take(4 * n * T * NA * KA);
    t.gpart = take(4 * (size_t)m->ks->grad_chunks(N) * m->lay.P);
    t.loss = take(8);
    t.total = o;
    return t;
}

template <class T>
T* at(void* base, size_t off) {
    return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

nep_status check_system(const nep_model* m, const nep_system* s) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (!s) return fail(NEP_ERR_ARG, "system is NULL");
    if (s->n_atoms < 0 || s->n_cfg < 1) return fail(NEP_ERR_ARG, "n_atoms < 0 or n_cfg < 1");
    if (!s->atom_off_host || !s->box_host) return fail(NEP_ERR_ARG, "host copies of atom_off/box are NULL");
    if (s->atom_off_host[0] != 0 || s->atom_off_host[s->n_cfg] != s->n_atoms)
        return fail(NEP_ERR_ARG, "atom_off must start at 0 and end at n_atoms");
    for (int b = 0; b < s->n_cfg; ++b) {
        if (s->atom_off_host[b + 1] < s->atom_off_host[b])
            return fail(NEP_ERR_ARG, "atom_off not non-decreasing at config %d", b);
        for (int d = 0; d < 3; ++d) {
            const float L = s->box_host[3 * b + d];
            if (!(L > 0.0f) || !std::isfinite(L))
                return fail(NEP_ERR_ARG, "box of config %d is not positive and finite", b);
        }
    }
    if (s->n_atoms > 0 && (!s->pos || !s->type)) return fail(NEP_ERR_ARG, "pos or type is NULL");
    if (!s->atom_off || !s->box) return fail(NEP_ERR_ARG, "atom_off or box is NULL");
    return NEP_OK;
}

nep_status check_nlist(const nep_nlist* nl, int N) {
    if (!nl) return fail(NEP_ERR_ARG, "neighbour list is NULL");
    if (nl->cap < 1 || nl->cap_ang < 1 || nl->cap_ang > nl->cap)
        return fail(NEP_ERR_ARG, "need 1 <= cap_ang <= cap (got cap=%d cap_ang=%d)", nl->cap, nl->cap_ang);
    if ((long long)nl->cap * N >= (1LL << 31))
        return fail(NEP_ERR_ARG, "cap * n_atoms must stay below 2^31");
    if ((long long)nl->cap_ang * N >= (1LL << 30))
        return fail(NEP_ERR_ARG, "cap_ang * n_atoms must stay below 2^30");
    if (N > 0 && (!nl->cnt || !nl->cnt_ang || !nl->nbr || !nl->rev || !nl->status))
        return fail(NEP_ERR_ARG, "neighbour list arrays are NULL");
    return NEP_OK;
}

bool boxes_allow_min_image(const nep_system* s, float rc_list) {
    for (int b = 0; b < s->n_cfg; ++b)
        for (int d = 0; d < 3; ++d)
            if (s->box_host[3 * b + d] < 2.0f * rc_list + 0.01f) return false;
    return true;
}

// size class of a system: log2 of its mean atoms per configuration
int size_bin(const nep_system* s) {
    const int mean = s->n_cfg > 0 ? s->n_atoms / s->n_cfg : 0;
    int b = 0;
    while ((1 << (b + 1)) <= mean && b + 1 < nep::kSizeBins) ++b;
    return b;
}

int angular_variant(const nep_model* m, const nep_system* s) {
    const int b = size_bin(s);
    return m->tune_angular[b] >= 0 ? m->tune_angular[b] : nep::kDefaultAngularVariant;
}
int radial_block(const nep_model* m, const nep_system* s) { return m->tune_radial[size_bin(s)]; }
int finish_block(const nep_model* m, const nep_system* s) { return m->tune_finish[size_bin(s)]; }
bool block_choice(int b) {
    for (int c : nep::kBlockChoices)
        if (b == c) return true;
    return false;
}

nep::EvalArgs make_args(const nep_model* m, const nep_system* s, const nep_nlist* nl, void* work,
                        const WsLayout& w) {
    nep::EvalArgs a;
    a.N = s->n_atoms;
    a.B = s->n_cfg;
    a.T = m->hp.n_types;
    a.H = m->hp.n_hidden;
    a.cap = nl->cap;
    a.cap_ang = nl->cap_ang;
    a.min_image = nl->min_image;
    a.rc_rad = m->hp.rc_rad;
    a.rc_ang = m->hp.rc_ang;
    a.pos4 = at<float4>(work, w.pos4);
    a.cfg = at<int>(work, w.cfg);
    a.box = s->box;
    a.cnt = nl->cnt;
    a.cnt_ang = nl->cnt_ang;
    a.nbr = nl->nbr;
    a.shift = nl->shift;
    a.rev = nl->rev;
    a.params = m->params;
    a.e_atom = at<float>(work, w.e_atom);
    a.fb = at<float>(work, w.fb);
    a.S = m->hp.precision ? at<float>(work, w.S) : nullptr;
    a.Pr = at<float>(work, w.Pr);
    a.comp = at<float4>(work, w.comp);
    a.cnt_comp = at<int>(work, w.cnt_comp);
    a.compr = nullptr;
    a.cnt_compr = nullptr;
    a.amask = at<unsigned long long>(work, w.amask);
    a.fin = at<float4>(work, w.fin);
    // the compact list of post-prefix entries inside rc_rad pays off only
    // when the list carries a shell beyond rc_rad (a skin)
    const bool use_rin = nl->skin > 0.0f;
    a.rin = use_rin ? at<int>(work, w.rin) : nullptr;
    a.rin_sh = use_rin && nl->shift ? at<int>(work, w.rin_sh) : nullptr;
    a.cnt_rin = use_rin ? at<int>(work, w.cnt_rin) : nullptr;
    a.fpart = at<float>(work, w.fpart);
    a.wat = at<float>(work, w.wat);
    a.status = nl->status;
    a.q_out = nullptr;
    a.p_out = nullptr;
    a.fb_out = nullptr;
    a.q16_kind = m->hp.precision;
    return a;
}

nep_status check_work(const nep_model* m, const nep_system* s, const nep_nlist* nl, void* work,
                      size_t work_bytes, WsLayout* w) {
    *w = ws_layout(m, s->n_atoms, s->n_cfg, nl->cap, nl->cap_ang);
    if (work_bytes < w->total)
        return fail(NEP_ERR_ARG, "workspace too small: %zu bytes given, %zu needed", work_bytes, w->total);
    if (!work && w->total) return fail(NEP_ERR_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return fail(NEP_ERR_ARG, "workspace must be 256-byte aligned");
    return NEP_OK;
}

// Scratch of the FP64 evaluation
struct Ws64Layout {
    size_t pos4, cfg, chunk_start, partial, prm, e, p, R, w;
    // training: FP64 forces, totals, adjoints, staged factors, gradient partials
    size_t force, etot, vir, lam, aE, mu, st, gpart;
    size_t total;
    int max_chunks;
};
Ws64Layout ws64_layout(const nep_model* m, int N, int B) {
    Ws64Layout w;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t n = (size_t)N;
    w.pos4 = take(16 * n);
    w.cfg = take(4 * n);
    w.chunk_start = take(4 * ((size_t)B + 1));
    w.max_chunks = (int)((n + nep::kChunk - 1) / nep::kChunk) + B;
    w.partial = take(80 * (size_t)w.max_chunks);
    w.prm = take(8 * (size_t)m->lay.P);
    w.e = take(8 * n);
    w.p = take(8 * n * m->hp.n_rad);
    w.R = take(8 * n * m->hp.n_ang * nep::kLM);
    w.w = take(72 * n);
    w.total = o;
    w.force = w.etot = w.vir = w.lam = w.aE = w.mu = w.st = w.gpart = 0;
    return w;
}
// the evaluation scratch followed by the training gradient's
Ws64Layout ws64_train_layout(const nep_model* m, int N, int B, int n_fields) {
    Ws64Layout w = ws64_layout(m, N, B);
    size_t o = w.total;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    const size_t n = (size_t)N;
    w.force = take(24 * n);
    w.etot = take(8 * (size_t)B);
    w.vir = take(72 * (size_t)B);
    w.lam = take(24 * n);
    w.aE = take(8 * (size_t)B);
    w.mu = take(72 * (size_t)B);
    w.st = take(8 * n * (size_t)n_fields);
    w.gpart = take(8 * (size_t)nep::fp64_grad_chunks(N) * (size_t)m->lay.P);
    w.total = o;
    return w;
}
// staged factors per atom of the FP64 gradient (the layout of nep_fp64.cu)
int fp64_fields_of(const nep_model* m) {
    nep::F64Args a{};
    a.D = m->lay.D;
    a.H = m->hp.n_hidden;
    a.NR = m->hp.n_rad;
    a.T = m->hp.n_types;
    a.KR = m->hp.k_rad;
    a.NA = m->hp.n_ang;
    a.KA = m->hp.k_ang;
    return nep::fp64_grad_fields(a);
}
bool fp64_grad_supported(const nep_hparams& hp) {
    return hp.n_types * hp.n_ang * hp.k_ang <= nep::kF64MaxBins;
}
bool fp64_supported(const nep_hparams& hp) {
    return hp.n_rad <= nep::kF64MaxN && hp.n_ang <= nep::kF64MaxN && hp.k_rad <= nep::kF64MaxK &&
           hp.k_ang <= nep::kF64MaxK;
}

// The generic FP32 evaluation (a model with no compiled kernel set): the
// FP64 path's two kernels in float, every pair term evaluated from both of
// its atoms, then the same FP64 sums.
nep_status efv_generic(nep_model* m, const nep_system* s, const nep_nlist* nl, float* e_atom, float* force,
                       double* e_tot, double* virial, void* work, const WsLayout& w, cudaStream_t st,
                       int n_owned) {
    const int N = s->n_atoms;
    nep::F32Args a{};
    a.N = N;
    a.B = s->n_cfg;
    a.T = m->hp.n_types;
    a.NR = m->hp.n_rad;
    a.NA = m->hp.n_ang;
    a.KR = m->hp.k_rad;
    a.KA = m->hp.k_ang;
    a.H = m->hp.n_hidden;
    a.H4 = m->hp.has_4body;
    a.D = m->lay.D;
    a.L = m->lay;
    a.rc_rad = m->hp.rc_rad;
    a.rc_ang = m->hp.rc_ang;
    a.pos = s->pos;
    a.type = s->type;
    a.cfg = at<int>(work, w.cfg);
    a.box = s->box;
    a.cnt = nl->cnt;
    a.nbr = nl->nbr;
    a.shift = nl->min_image ? nullptr : nl->shift;
    a.prm = m->params;
    a.e = e_atom ? e_atom : at<float>(work, w.e_atom);
    a.p = at<float>(work, w.gen_p);
    a.R = at<float>(work, w.gen_R);
    a.w = at<float>(work, w.gen_w);
    a.force = force;
    a.atom_off = s->atom_off;
    a.chunk_start = at<int>(work, w.chunk_start);
    a.partial = at<double>(work, w.partial);
    a.n_owned = n_owned < 0 ? N : n_owned;
    const int nt = m->n_timing;
    m->n_timing = 0;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (nt) NEP_CUDA(cudaStreamIsCapturing(st, &cap), "capture status");
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (nt) NEP_CUDA(cudaEventRecordWithFlags(m->timing[0], st, rec_flags), "timing event");
    NEP_CUDA(nep::launch_efv_generic(a, w.max_chunks, e_tot, virial, st), "generic FP32 kernels");
    for (int k = 1; k < 4 && nt; ++k) NEP_CUDA(cudaEventRecordWithFlags(m->timing[k], st, rec_flags), "timing event");
    return NEP_OK;
}

nep_status efv_impl(nep_model* m, const nep_system* s, const nep_nlist* nl, float* e_atom,
                    float* force, double* e_tot, double* virial, void* work, const WsLayout& w,
                    cudaStream_t st, int n_owned = -1) {
    const int N = s->n_atoms, B = s->n_cfg;
    NEP_CUDA(nep::launch_pack(s->pos, s->type, s->atom_off, N, B, m->hp.n_types, at<float4>(work, w.pos4),
                              at<int>(work, w.cfg), nl->status, st),
             "pack");
    NEP_CUDA(nep::launch_chunk_plan(s->atom_off, B, at<int>(work, w.chunk_start), st), "chunk plan");
    if (!m->ks) return efv_generic(m, s, nl, e_atom, force, e_tot, virial, work, w, st, n_owned);
    const nep::EvalArgs a = make_args(m, s, nl, work, w);
    const int vd = angular_variant(m, s);
    const int nt = m->n_timing;
    m->n_timing = 0;
    // inside stream capture an event record must be marked external to become
    // a timing node of the graph; outside capture the flag is not accepted
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (nt) NEP_CUDA(cudaStreamIsCapturing(st, &cap), "capture status");
    const unsigned rec_flags = cap == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    auto mark = [&](int k) -> cudaError_t {
        return nt ? cudaEventRecordWithFlags(m->timing[k], st, rec_flags) : cudaSuccess;
    };
    NEP_CUDA(mark(0), "timing event");
    if (N > 0) NEP_CUDA(m->ks->radial(a, st, radial_block(m, s)), "radial kernel");
    NEP_CUDA(mark(1), "timing event");
    if (N > 0) NEP_CUDA(m->ks->angular(a, st, vd), "angular kernel");
    NEP_CUDA(mark(2), "timing event");
    nep::FinishArgs f;
    f.atom_off = s->atom_off;
    f.chunk_start = at<int>(work, w.chunk_start);
    f.partial = at<double>(work, w.partial);
    f.force = force;
    f.e_out = e_atom;
    f.n_owned = n_owned < 0 ? N : n_owned;
    NEP_CUDA(m->ks->finish(a, f, w.max_chunks, st, finish_block(m, s)), "finish kernel");
    NEP_CUDA(mark(3), "timing event");
    NEP_CUDA(nep::launch_final_reduce(B, at<int>(work, w.chunk_start), at<double>(work, w.partial), e_tot,
                                      virial, st),
             "final reduce");
    return NEP_OK;
}

nep_status train_impl(nep_model* m, const nep_system* s, const nep_nlist* nl, const double* e_lbl,
                      const float* f_lbl, const double* v_lbl, const float* w_host, int loss_mode,
                      const double* a_e, const float* lam, const double* mu, float* grad,
                      double* loss, void* work, const TrainLayout& tl, cudaStream_t st) {
    const int N = s->n_atoms, B = s->n_cfg;
    const WsLayout& w = tl.w;
    NEP_CUDA(nep::launch_pack(s->pos, s->type, s->atom_off, N, B, m->hp.n_types, at<float4>(work, w.pos4),
                              at<int>(work, w.cfg), nl->status, st),
             "pack");
    NEP_CUDA(nep::launch_chunk_plan(s->atom_off, B, at<int>(work, w.chunk_start), st), "chunk plan");
    nep::EvalArgs a = make_args(m, s, nl, work, w);
    a.q16_kind = 0;
    a.S = at<float>(work, w.S);
    a.compr = at<float4>(work, tl.compr);
    a.cnt_compr = at<int>(work, tl.cnt_compr);
    a.q_out = at<float>(work, tl.q);
    a.p_out = at<float>(work, tl.p);
    a.fb_out = a.fb;
    const int vd = angular_variant(m, s);
    if (N > 0) NEP_CUDA(m->ks->radial(a, st, 0), "radial kernel");
    if (N > 0) NEP_CUDA(m->ks->angular(a, st, vd), "angular kernel");
    if (e_lbl) {
        // forward forces, energies and virials, then the loss and its adjoints
        nep::FinishArgs f;
        f.atom_off = s->atom_off;
        f.chunk_start = at<int>(work, w.chunk_start);
        f.partial = at<double>(work, w.partial);
        f.force = at<float>(work, tl.force);
        f.e_out = nullptr;
        f.n_owned = N;
        NEP_CUDA(m->ks->finish(a, f, w.max_chunks, st, 0), "finish kernel");
        NEP_CUDA(nep::launch_final_reduce(B, at<int>(work, w.chunk_start), at<double>(work, w.partial),
                                          at<double>(work, tl.etot), at<double>(work, tl.vir), st),
                 "final reduce");
        NEP_CUDA(nep::launch_loss(N, B, s->atom_off, at<int>(work, w.chunk_start), w.max_chunks,
                                  at<float>(work, tl.force), f_lbl, at<double>(work, tl.etot),
                                  at<double>(work, tl.vir), e_lbl, v_lbl, w_host, loss_mode,
                                  at<float4>(work, tl.lam4), at<float>(work, tl.aE),
                                  at<float>(work, tl.mu), at<double>(work, tl.partialF),
                                  loss ? loss : at<double>(work, tl.loss), st),
                 "loss");
    } else {
        NEP_CUDA(nep::launch_pack_adjoint(N, B, lam, a_e, mu, at<float4>(work, tl.lam4),
                                          at<float>(work, tl.aE), at<float>(work, tl.mu), st),
                 "adjoints");
    }
    nep::TrainArgs t;
    t.e = a;
    t.lam4 = at<float4>(work, tl.lam4);
    t.aE = at<float>(work, tl.aE);
    t.mu = at<float>(work, tl.mu);
    t.dq = at<float>(work, tl.dq);
    t.dS = at<float>(work, tl.dS);
    t.df = at<float>(work, tl.df);
    t.coef = at<float>(work, tl.coef);
    t.rho = at<float>(work, tl.rho);
    t.xz = at<float>(work, tl.xz);
    t.bins = at<float>(work, tl.bins);
    t.gpart = at<float>(work, tl.gpart);
    t.grad = grad;
    NEP_CUDA(m->ks->train(t, st), "gradient kernels");
    return NEP_OK;
}

nep_status check_train_work(const nep_model* m, const nep_system* s, const nep_nlist* nl, void* work,
                            size_t work_bytes, TrainLayout* tl) {
    *tl = train_layout(m, s->n_atoms, s->n_cfg, nl->cap, nl->cap_ang);
    if (work_bytes < tl->total)
        return fail(NEP_ERR_ARG, "training workspace too small: %zu bytes given, %zu needed "
                    "(nep_train_workspace_bytes)", work_bytes, tl->total);
    if (!work) return fail(NEP_ERR_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return fail(NEP_ERR_ARG, "workspace must be 256-byte aligned");
    return NEP_OK;
}

nep_status neighbors_impl(nep_model* m, const nep_system* s, float skin, nep_nlist* nl, void* work,
                          const WsLayout& w, cudaStream_t st) {
    const int N = s->n_atoms, B = s->n_cfg;
    const float rc_list = m->hp.rc_rad + skin;
    const float rc_list_ang = m->hp.rc_ang + skin;
    const bool mi = boxes_allow_min_image(s, rc_list);
    if (!mi && !nl->shift)
        return fail(NEP_ERR_ARG,
                    "a box edge is shorter than 2*(rc+skin)+0.01; the list needs a shift array");
    nl->skin = skin;
    nl->min_image = mi ? 1 : 0;
    NEP_CUDA(cudaMemsetAsync(nl->status, 0, 4 * sizeof(int), st), "clear status");
    NEP_CUDA(nep::launch_pack(s->pos, s->type, s->atom_off, N, B, m->hp.n_types, at<float4>(work, w.pos4),
                              at<int>(work, w.cfg), nl->status, st),
             "pack");
    nep::NbrWork nw;
    nw.plan = at<nep::CellPlan>(work, w.plan);
    nw.cell_of = at<int>(work, w.cell_of);
    nw.rank = at<int>(work, w.rank);
    nw.cell_cnt = at<int>(work, w.cell_cnt);
    nw.cell_start = at<int>(work, w.cell_start);
    nw.cell_atoms = at<int>(work, w.cell_atoms);
    nw.cell_pos = at<float4>(work, w.cell_pos);
    nw.scan_tmp = at<int>(work, w.scan_tmp);
    nw.shell = at<int2>(work, w.shell);
    nw.row_start = at<unsigned char>(work, w.row_start);
    nw.slot_row = at<unsigned char>(work, w.slot_row);
    nw.cmax = w.cmax;
    nep_nlist copy = *nl;
    if (mi) copy.shift = nullptr;
    NEP_CUDA(nep::launch_neighbors(s->pos, at<float4>(work, w.pos4), s->atom_off, s->box, at<int>(work, w.cfg), N, B, rc_list,
                                   rc_list_ang, m->hp.rc_rad, mi ? 1 : 0, &copy, nw, st),
             "neighbour build");
    return NEP_OK;
}

}  // namespace

extern "C" {

const char* nep_version(void) { return "libnep 0.1 (sm_103a)"; }

const char* nep_last_error(void) { return g_err.c_str(); }

size_t nep_num_params(const nep_hparams* hp) {
    if (!hp_valid(hp)) return 0;
    const nep::ParamLayout L = nep::param_layout(hp->n_types, hp->n_rad, hp->n_ang, hp->k_rad,
                                                 hp->k_ang, hp->has_4body, hp->n_hidden);
    return (size_t)L.P;
}

int nep_supported(const nep_hparams* hp) {
    if (!hp_valid(hp)) return 0;
    if (hp->precision != 0 && hp->n_hidden > nep::kTcMaxHidden) return 0;
    if (nep::find_kernel_set(hp->n_rad, hp->n_ang, hp->k_rad, hp->k_ang, hp->has_4body, hp->n_types))
        return 1;
    return hp->precision == 0 && fp64_supported(*hp) ? 2 : 0;
}

nep_status nep_create(const nep_hparams* hp, const float* params_host, size_t n_params,
                      nep_model** out) {
    if (!out) return fail(NEP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!hp_valid(hp)) return fail(NEP_ERR_ARG, "invalid hyper-parameters (l_max must be 4, 1 <= n_types <= 4, rc_ang <= rc_rad)");
    const nep::KernelSet* ks = nep::find_kernel_set(hp->n_rad, hp->n_ang, hp->k_rad, hp->k_ang,
                                                    hp->has_4body, hp->n_types);
    if (!ks && (hp->precision != 0 || !fp64_supported(*hp)))
        return fail(NEP_ERR_UNSUPPORTED,
                    "no kernel compiled for n_rad=%d n_ang=%d k_rad=%d k_ang=%d 4body=%d types=%d, and the "
                    "generic path takes FP32 only with n_rad, n_ang <= %d and k_rad, k_ang <= %d",
                    hp->n_rad, hp->n_ang, hp->k_rad, hp->k_ang, hp->has_4body, hp->n_types, nep::kF64MaxN,
                    nep::kF64MaxK);
    if (hp->precision != 0 && hp->n_hidden > nep::kTcMaxHidden)
        return fail(NEP_ERR_UNSUPPORTED, "the FP16/BF16 network supports n_hidden <= %d", nep::kTcMaxHidden);
    const size_t P = nep_num_params(hp);
    if (n_params != P) return fail(NEP_ERR_ARG, "expected %zu parameters, got %zu", P, n_params);
    if (!params_host) return fail(NEP_ERR_ARG, "params_host is NULL");
    for (size_t k = 0; k < P; ++k)
        if (!std::isfinite(params_host[k])) return fail(NEP_ERR_ARG, "parameter %zu is not finite", k);
    nep_model* m = new nep_model();
    m->hp = *hp;
    m->ks = ks;
    m->lay = nep::param_layout(hp->n_types, hp->n_rad, hp->n_ang, hp->k_rad, hp->k_ang,
                               hp->has_4body, hp->n_hidden);
    cudaGetDevice(&m->device);
    m->n_timing = 0;
    for (int b = 0; b < nep::kSizeBins; ++b) {
        m->tune_angular[b] = -1;
        m->tune_radial[b] = 0;
        m->tune_finish[b] = 0;
    }
    cudaError_t e = ks ? ks->init(hp->n_hidden) : cudaSuccess;
    if (e == cudaSuccess && ks) e = ks->train_init(hp->n_hidden);
    if (e != cudaSuccess) {
        delete m;
        return cuda_fail(e, "kernel attributes");
    }
    e = cudaMalloc(&m->params, sizeof(float) * P);
    if (e != cudaSuccess) {
        delete m;
        return fail(NEP_ERR_NOMEM, "cudaMalloc of %zu parameters: %s", P, cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->params, params_host, sizeof(float) * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->params);
        delete m;
        return cuda_fail(e, "copy parameters");
    }
    *out = m;
    return NEP_OK;
}

nep_status nep_destroy(nep_model* m) {
    if (!m) return NEP_OK;
    cudaError_t e = cudaFree(m->params);
    delete m;
    if (e != cudaSuccess) return cuda_fail(e, "free parameters");
    return NEP_OK;
}

nep_status nep_get_params(const nep_model* m, float* params_dev, void* stream) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (!params_dev) return fail(NEP_ERR_ARG, "params_dev is NULL");
    NEP_CUDA(cudaMemcpyAsync(params_dev, m->params, sizeof(float) * nep_num_params(&m->hp),
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
             "copy parameters");
    return NEP_OK;
}

nep_status nep_set_params(nep_model* m, const float* params_dev, void* stream) {
    if (!m || !params_dev) return fail(NEP_ERR_ARG, "model or params is NULL");
    NEP_CUDA(cudaMemcpyAsync(m->params, params_dev, sizeof(float) * (size_t)m->lay.P,
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream),
             "set params");
    return NEP_OK;
}

size_t nep_workspace_bytes(const nep_model* m, int n_atoms, int n_cfg, int cap, int cap_ang) {
    if (!m || n_atoms < 0 || n_cfg < 1 || cap < 1 || cap_ang < 1) return 0;
    return ws_layout(m, n_atoms, n_cfg, cap, cap_ang).total;
}

nep_status nep_neighbors(nep_model* m, const nep_system* sys, float skin, nep_nlist* nl, void* work,
                         size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!(skin >= 0.0f) || !std::isfinite(skin)) return fail(NEP_ERR_ARG, "skin must be finite and >= 0");
    WsLayout w;
    if ((s = check_work(m, sys, nl, work, work_bytes, &w)) != NEP_OK) return s;
    return neighbors_impl(m, sys, skin, nl, work, w, (cudaStream_t)stream);
}

nep_status nep_energy_forces_virial(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                    float* e_atom, float* force, double* e_tot, double* virial,
                                    void* work, size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (sys->n_atoms > 0 && !force) return fail(NEP_ERR_ARG, "force is NULL");
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built (no shifts, not min-image)");
    WsLayout w;
    if ((s = check_work(m, sys, nl, work, work_bytes, &w)) != NEP_OK) return s;
    return efv_impl(m, sys, nl, e_atom, force, e_tot, virial, work, w, (cudaStream_t)stream);
}

size_t nep_workspace_bytes_fp64(const nep_model* m, int n_atoms, int n_cfg) {
    if (!m || n_atoms < 0 || n_cfg < 1) return 0;
    return ws64_layout(m, n_atoms, n_cfg).total;
}

size_t nep_train_workspace_bytes_fp64(const nep_model* m, int n_atoms, int n_cfg) {
    if (!m || n_atoms < 0 || n_cfg < 1) return 0;
    return ws64_train_layout(m, n_atoms, n_cfg, fp64_fields_of(m)).total;
}

}  // extern "C"

namespace {
// checks shared by the FP64 calls, then the packed positions, the chunk plan
// and (params == NULL) the promoted parameters
nep_status fp64_begin(nep_model* m, const nep_system* sys, const nep_nlist* nl, const double* params,
                      void* work, size_t work_bytes, const Ws64Layout& w, cudaStream_t st, nep::F64Args* out) {
    nep_status s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!fp64_supported(m->hp))
        return fail(NEP_ERR_UNSUPPORTED, "the FP64 path supports n_rad, n_ang <= %d and k_rad, k_ang <= %d",
                    nep::kF64MaxN, nep::kF64MaxK);
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built (no shifts, not min-image)");
    if (work_bytes < w.total)
        return fail(NEP_ERR_ARG, "workspace too small: %zu bytes given, %zu needed", work_bytes, w.total);
    if (!work && w.total) return fail(NEP_ERR_ARG, "workspace is NULL");
    if ((reinterpret_cast<uintptr_t>(work) & 255) != 0)
        return fail(NEP_ERR_ARG, "workspace must be 256-byte aligned");
    const int N = sys->n_atoms, B = sys->n_cfg;
    NEP_CUDA(nep::launch_pack(sys->pos, sys->type, sys->atom_off, N, B, m->hp.n_types, at<float4>(work, w.pos4),
                              at<int>(work, w.cfg), nl->status, st),
             "pack");
    NEP_CUDA(nep::launch_chunk_plan(sys->atom_off, B, at<int>(work, w.chunk_start), st), "chunk plan");
    if (!params) {
        NEP_CUDA(nep::launch_promote(m->params, at<double>(work, w.prm), m->lay.P, st), "promote parameters");
        params = at<double>(work, w.prm);
    }
    nep::F64Args a{};
    a.N = N;
    a.B = B;
    a.T = m->hp.n_types;
    a.NR = m->hp.n_rad;
    a.NA = m->hp.n_ang;
    a.KR = m->hp.k_rad;
    a.KA = m->hp.k_ang;
    a.H = m->hp.n_hidden;
    a.H4 = m->hp.has_4body;
    a.D = m->lay.D;
    a.L = m->lay;
    a.rc_rad = (double)m->hp.rc_rad;
    a.rc_ang = (double)m->hp.rc_ang;
    a.pos = sys->pos;
    a.type = sys->type;
    a.cfg = at<int>(work, w.cfg);
    a.box = sys->box;
    a.cnt = nl->cnt;
    a.nbr = nl->nbr;
    a.shift = nl->min_image ? nullptr : nl->shift;
    a.prm = params;
    a.e = at<double>(work, w.e);
    a.p = at<double>(work, w.p);
    a.R = at<double>(work, w.R);
    a.w = at<double>(work, w.w);
    a.atom_off = sys->atom_off;
    a.chunk_start = at<int>(work, w.chunk_start);
    a.partial = at<double>(work, w.partial);
    a.n_owned = N;
    *out = a;
    return NEP_OK;
}
}  // namespace

extern "C" {

nep_status nep_energy_forces_virial_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                         const double* params, double* e_atom, double* force,
                                         double* e_tot, double* virial, void* work, size_t work_bytes,
                                         void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if (sys->n_atoms > 0 && !force) return fail(NEP_ERR_ARG, "force is NULL");
    const Ws64Layout w = ws64_layout(m, sys->n_atoms, sys->n_cfg);
    nep::F64Args a;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = fp64_begin(m, sys, nl, params, work, work_bytes, w, st, &a)) != NEP_OK) return s;
    if (e_atom) a.e = e_atom;
    a.force = force;
    NEP_CUDA(nep::launch_efv_fp64(a, w.max_chunks, e_tot, virial, st), "FP64 kernels");
    return NEP_OK;
}

nep_status nep_param_grad_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl, const double* params,
                               const double* e_lbl, const double* f_lbl, const double* v_lbl,
                               const float* w_host, int loss_mode, double* grad, double* loss, void* work,
                               size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if (!fp64_grad_supported(m->hp))
        return fail(NEP_ERR_UNSUPPORTED, "the FP64 gradient supports n_types * n_ang * k_ang <= %d",
                    nep::kF64MaxBins);
    if (!grad) return fail(NEP_ERR_ARG, "grad is NULL");
    if (!e_lbl || !v_lbl || (sys->n_atoms > 0 && !f_lbl)) return fail(NEP_ERR_ARG, "labels are NULL");
    if (!w_host) return fail(NEP_ERR_ARG, "w_host is NULL");
    if (loss_mode != 0 && loss_mode != 1) return fail(NEP_ERR_ARG, "loss_mode must be 0 or 1");
    const Ws64Layout w = ws64_train_layout(m, sys->n_atoms, sys->n_cfg, fp64_fields_of(m));
    nep::F64Args a;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = fp64_begin(m, sys, nl, params, work, work_bytes, w, st, &a)) != NEP_OK) return s;
    a.force = at<double>(work, w.force);
    double* etot = at<double>(work, w.etot);
    double* vir = at<double>(work, w.vir);
    NEP_CUDA(nep::launch_efv_fp64(a, w.max_chunks, etot, vir, st), "FP64 kernels");
    double* lam = at<double>(work, w.lam);
    double* aE = at<double>(work, w.aE);
    double* mu = at<double>(work, w.mu);
    NEP_CUDA(nep::launch_loss_fp64(a, w.max_chunks, etot, vir, e_lbl, f_lbl, v_lbl, w_host, loss_mode, lam, aE,
                                   mu, loss, st),
             "FP64 loss");
    a.lam = lam;
    a.aE = aE;
    a.mu = mu;
    a.st = at<double>(work, w.st);
    a.gpart = at<double>(work, w.gpart);
    a.grad = grad;
    NEP_CUDA(nep::launch_grad_fp64(a, st), "FP64 gradient");
    return NEP_OK;
}

nep_status nep_param_grad_adjoint_fp64(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                       const double* params, const double* a_e, const double* lam,
                                       const double* mu, double* grad, void* work, size_t work_bytes,
                                       void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if (!fp64_grad_supported(m->hp))
        return fail(NEP_ERR_UNSUPPORTED, "the FP64 gradient supports n_types * n_ang * k_ang <= %d",
                    nep::kF64MaxBins);
    if (!grad) return fail(NEP_ERR_ARG, "grad is NULL");
    if (!a_e || !mu || (sys->n_atoms > 0 && !lam)) return fail(NEP_ERR_ARG, "adjoints are NULL");
    const Ws64Layout w = ws64_train_layout(m, sys->n_atoms, sys->n_cfg, fp64_fields_of(m));
    nep::F64Args a;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = fp64_begin(m, sys, nl, params, work, work_bytes, w, st, &a)) != NEP_OK) return s;
    a.lam = lam;
    a.aE = a_e;
    a.mu = mu;
    a.st = at<double>(work, w.st);
    a.gpart = at<double>(work, w.gpart);
    a.grad = grad;
    NEP_CUDA(nep::launch_grad_fp64(a, st), "FP64 gradient");
    return NEP_OK;
}

nep_status nep_energy_forces_virial_owned(nep_model* m, const nep_system* sys, const nep_nlist* nl, int n_owned,
                                          float* e_atom, float* force, double* e_tot, double* virial, void* work,
                                          size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (n_owned < 0 || n_owned > sys->n_atoms) return fail(NEP_ERR_ARG, "need 0 <= n_owned <= n_atoms");
    if (sys->n_atoms > 0 && !force) return fail(NEP_ERR_ARG, "force is NULL");
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built (no shifts, not min-image)");
    WsLayout w;
    if ((s = check_work(m, sys, nl, work, work_bytes, &w)) != NEP_OK) return s;
    return efv_impl(m, sys, nl, e_atom, force, e_tot, virial, work, w, (cudaStream_t)stream, n_owned);
}

size_t nep_domain_workspace_bytes(int n_atoms) {
    return n_atoms < 0 ? 0 : nep::domain_scratch_bytes(n_atoms);
}

nep_status nep_domain_select(const float* pos, int n_atoms, const float* box_host, float x_lo, float x_hi,
                             float halo, int* idx, int* img, int cap, int* counts, void* work, size_t work_bytes,
                             void* stream) {
    if (n_atoms < 0 || cap < 0) return fail(NEP_ERR_ARG, "n_atoms and cap must be >= 0");
    if (!box_host || !counts || (n_atoms > 0 && !pos) || (cap > 0 && (!idx || !img)))
        return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    const float Lx = box_host[0];
    if (!(Lx > 0.0f) || !std::isfinite(Lx)) return fail(NEP_ERR_ARG, "box x must be positive and finite");
    if (!(x_lo >= 0.0f && x_lo < x_hi && x_hi <= Lx)) return fail(NEP_ERR_ARG, "need 0 <= x_lo < x_hi <= box x");
    if (!(halo >= 0.0f) || !(x_hi - x_lo + 2.0f * halo <= Lx))
        return fail(NEP_ERR_ARG, "need halo >= 0 and slab + 2 halo <= box x (one image per atom)");
    if (work_bytes < nep::domain_scratch_bytes(n_atoms) || !work)
        return fail(NEP_ERR_ARG, "workspace too small: %zu bytes given, %zu needed", work_bytes,
                    nep::domain_scratch_bytes(n_atoms));
    NEP_CUDA(nep::launch_domain_select(pos, n_atoms, Lx, x_lo, x_hi, halo, idx, img, cap, counts, work,
                                       (cudaStream_t)stream),
             "domain select");
    return NEP_OK;
}

nep_status nep_domain_gather(const float* pos, const int* type, int n_atoms, const int* idx, const int* img,
                             int n_local, const float* box_host, float x_origin, float* pos_local, int* type_local,
                             void* stream) {
    if (n_atoms < 0 || n_local < 0) return fail(NEP_ERR_ARG, "sizes must be >= 0");
    if (!box_host || (n_local > 0 && (!pos || !type || !idx || !img || !pos_local || !type_local)))
        return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    NEP_CUDA(nep::launch_domain_gather(pos, type, n_atoms, idx, img, n_local, box_host[0], x_origin, pos_local,
                                       type_local, (cudaStream_t)stream),
             "domain gather");
    return NEP_OK;
}

nep_status nep_domain_band(const float* pos, int n_atoms, float x_lo, float x_hi, int* idx, int cap, int* counts,
                           void* work, size_t work_bytes, void* stream) {
    if (n_atoms < 0 || cap < 0) return fail(NEP_ERR_ARG, "n_atoms and cap must be >= 0");
    if (!counts || (n_atoms > 0 && !pos) || (cap > 0 && !idx)) return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    if (!(x_lo < x_hi) || std::isnan(x_lo) || std::isnan(x_hi)) return fail(NEP_ERR_ARG, "need x_lo < x_hi");
    if (work_bytes < nep::domain_scratch_bytes(n_atoms) || !work)
        return fail(NEP_ERR_ARG, "workspace too small: %zu bytes given, %zu needed", work_bytes,
                    nep::domain_scratch_bytes(n_atoms));
    // the slab selection with no halo: every atom in [x_lo, x_hi) is "owned", none is a ghost
    NEP_CUDA(nep::launch_domain_select(pos, n_atoms, 1.0f, x_lo, x_hi, 0.0f, idx, nullptr, cap, counts, work,
                                       (cudaStream_t)stream),
             "domain band");
    return NEP_OK;
}

nep_status nep_domain_take(const void* src, int n_src, int ncomp, const int* idx, int n, void* dst, void* stream) {
    if (n_src < 0 || n < 0 || ncomp < 1) return fail(NEP_ERR_ARG, "need n_src, n >= 0 and ncomp >= 1");
    if (n > 0 && (!src || !idx || !dst)) return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    NEP_CUDA(nep::launch_domain_take(src, n_src, ncomp, idx, n, dst, (cudaStream_t)stream), "domain take");
    return NEP_OK;
}

nep_status nep_domain_place(const void* src, int n, int ncomp, float box_x, float x_center, float x_origin,
                            void* dst, int dst_stride, int dst_offset, void* stream) {
    if (n < 0 || ncomp < 1 || dst_offset < 0 || (long long)dst_offset + n > dst_stride)
        return fail(NEP_ERR_ARG, "need n >= 0, ncomp >= 1 and 0 <= dst_offset, dst_offset + n <= dst_stride");
    if (!std::isfinite(box_x) || !std::isfinite(x_center) || !std::isfinite(x_origin))
        return fail(NEP_ERR_ARG, "box_x, x_center and x_origin must be finite");
    if (n > 0 && (!src || !dst)) return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    NEP_CUDA(nep::launch_domain_place(src, n, ncomp, box_x, x_center, x_origin, dst, dst_stride, dst_offset,
                                      (cudaStream_t)stream),
             "domain place");
    return NEP_OK;
}

nep_status nep_domain_scatter(const float* src, int n_local, int ncomp, const int* idx, int n_owned, float* dst,
                              int n_atoms, void* stream) {
    if (n_local < 0 || n_owned < 0 || n_owned > n_local || ncomp < 1 || n_atoms < 0)
        return fail(NEP_ERR_ARG, "need 0 <= n_owned <= n_local and ncomp >= 1");
    if (n_owned > 0 && (!src || !idx || !dst)) return fail(NEP_ERR_ARG, "a pointer argument is NULL");
    NEP_CUDA(nep::launch_domain_scatter(src, n_local, ncomp, idx, n_owned, dst, n_atoms, (cudaStream_t)stream),
             "domain scatter");
    return NEP_OK;
}

nep_status nep_md_kick(nep_model* m, const nep_system* sys, float* vel, const float* force, const float* masses_host,
                       float half_dt, float drift_dt, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if (!masses_host) return fail(NEP_ERR_ARG, "masses_host is NULL");
    if (sys->n_atoms > 0 && (!vel || !force)) return fail(NEP_ERR_ARG, "vel or force is NULL");
    if (!std::isfinite(half_dt) || !(drift_dt >= 0.0f) || !std::isfinite(drift_dt))
        return fail(NEP_ERR_ARG, "half_dt must be finite and drift_dt finite and >= 0");
    float inv_m[nep::kMaxTypes] = {0, 0, 0, 0};
    for (int t = 0; t < m->hp.n_types; ++t) {
        if (!(masses_host[t] > 0.0f)) return fail(NEP_ERR_ARG, "mass of species %d must be positive", t);
        inv_m[t] = 1.0f / (masses_host[t] * 103.6427f);
    }
    float* pos = drift_dt > 0.0f ? const_cast<float*>(sys->pos) : nullptr;
    NEP_CUDA(nep::launch_kick(vel, force, sys->type, inv_m, sys->n_atoms, half_dt, pos, drift_dt,
                              (cudaStream_t)stream),
             "kick");
    return NEP_OK;
}

nep_status nep_md_wrap(nep_model* m, const nep_system* sys, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    NEP_CUDA(nep::launch_wrap_segments(const_cast<float*>(sys->pos), sys->atom_off, sys->n_cfg, sys->box,
                                       sys->n_atoms, (cudaStream_t)stream),
             "wrap");
    return NEP_OK;
}

nep_status nep_md_step(nep_model* m, const nep_system* sys, nep_nlist* nl, float* vel, float* force,
                       double* e_tot, double* virial, const float* masses_host, float dt, float skin,
                       int rebuild, void* work, size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!masses_host) return fail(NEP_ERR_ARG, "masses_host is NULL");
    if (sys->n_atoms > 0 && (!vel || !force)) return fail(NEP_ERR_ARG, "vel or force is NULL");
    if (!(dt > 0.0f) || !std::isfinite(dt)) return fail(NEP_ERR_ARG, "dt must be positive");
    WsLayout w;
    if ((s = check_work(m, sys, nl, work, work_bytes, &w)) != NEP_OK) return s;
    float inv_m[nep::kMaxTypes] = {0, 0, 0, 0};
    for (int t = 0; t < m->hp.n_types; ++t) {
        if (!(masses_host[t] > 0.0f)) return fail(NEP_ERR_ARG, "mass of species %d must be positive", t);
        inv_m[t] = 1.0f / (masses_host[t] * 103.6427f);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int N = sys->n_atoms;
    float* pos = const_cast<float*>(sys->pos);
    NEP_CUDA(nep::launch_kick(vel, force, sys->type, inv_m, N, 0.5f * dt, pos, dt, st), "kick/drift");
    if (rebuild) {
        NEP_CUDA(nep::launch_pack(sys->pos, sys->type, sys->atom_off, N, sys->n_cfg, m->hp.n_types,
                                  at<float4>(work, w.pos4), at<int>(work, w.cfg), nl->status, st),
                 "pack");
        NEP_CUDA(nep::launch_wrap(pos, at<int>(work, w.cfg), sys->box, N, st), "wrap");
        if ((s = neighbors_impl(m, sys, skin, nl, work, w, st)) != NEP_OK) return s;
    } else if (!nl->min_image && !nl->shift) {
        return fail(NEP_ERR_STATE, "list was not built");
    }
    if ((s = efv_impl(m, sys, nl, nullptr, force, e_tot, virial, work, w, st)) != NEP_OK) return s;
    NEP_CUDA(nep::launch_kick(vel, force, sys->type, inv_m, N, 0.5f * dt, nullptr, 0.0f, st), "kick");
    return NEP_OK;
}

}  // extern "C"

// Scratch of nep_energy_forces_virial_noalloc: one fixed device array per
// GPU, created when the module loads and never freed before exit.  In host
// code g_noalloc_scratch names a host-side stand-in, not device memory, so
// its device address is looked up per device and passed to the kernels.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NEP_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

nep_status noalloc_scratch(void** out) {
    int dev = 0;
    NEP_CUDA(cudaGetDevice(&dev), "current device");
    if (dev < 0 || dev >= kMaxDevices) return fail(NEP_ERR_ARG, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        NEP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch), "address of the static scratch array");
        if (!p) return fail(NEP_ERR_CUDA, "static scratch array has no device address");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return NEP_OK;
}
}  // namespace

extern "C" {

nep_status nep_energy_forces_virial_noalloc(nep_model* m, const nep_system* sys,
                                            const nep_nlist* nl, float* e_atom, float* force,
                                            double* e_tot, double* virial, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (sys->n_atoms > 0 && !force) return fail(NEP_ERR_ARG, "force is NULL");
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built (no shifts, not min-image)");
    const WsLayout w = ws_layout(m, sys->n_atoms, sys->n_cfg, nl->cap, nl->cap_ang);
    if (w.total > NEP_NOALLOC_SCRATCH_BYTES)
        return fail(NEP_ERR_ARG,
                    "system needs %zu bytes of scratch, the static array holds %zu "
                    "(use nep_energy_forces_virial with a caller workspace)",
                    w.total, (size_t)NEP_NOALLOC_SCRATCH_BYTES);
    void* work = nullptr;
    if ((s = noalloc_scratch(&work)) != NEP_OK) return s;
    return efv_impl(m, sys, nl, e_atom, force, e_tot, virial, work, w, (cudaStream_t)stream);
}

size_t nep_train_workspace_bytes(const nep_model* m, int n_atoms, int n_cfg, int cap, int cap_ang) {
    if (!m || n_atoms < 0 || n_cfg < 1 || cap < 1 || cap_ang < 1) return 0;
    // a generic model has no FP32 training operator: its evaluation scratch only
    if (!m->ks) return ws_layout(m, n_atoms, n_cfg, cap, cap_ang).total;
    return train_layout(m, n_atoms, n_cfg, cap, cap_ang).total;
}

nep_status nep_param_grad(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                          const double* e_lbl, const float* f_lbl, const double* v_lbl,
                          const float* w_host, int loss_mode, float* grad, double* loss, void* work,
                          size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!e_lbl || !v_lbl || (sys->n_atoms > 0 && !f_lbl)) return fail(NEP_ERR_ARG, "labels are NULL");
    if (!w_host) return fail(NEP_ERR_ARG, "loss weights are NULL");
    if (loss_mode != 0 && loss_mode != 1) return fail(NEP_ERR_ARG, "loss_mode must be 0 or 1");
    if (!grad) return fail(NEP_ERR_ARG, "grad is NULL");
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built");
    if (m->hp.precision != 0)
        return fail(NEP_ERR_UNSUPPORTED, "the gradient is computed for FP32 models (precision 0)");
    if (!m->ks)
        return fail(NEP_ERR_UNSUPPORTED, "no FP32 training operator for this model's shape (generic path): "
                                         "use nep_param_grad_fp64");
    TrainLayout tl;
    if ((s = check_train_work(m, sys, nl, work, work_bytes, &tl)) != NEP_OK) return s;
    return train_impl(m, sys, nl, e_lbl, f_lbl, v_lbl, w_host, loss_mode, nullptr, nullptr, nullptr, grad,
                      loss, work, tl, (cudaStream_t)stream);
}

nep_status nep_param_grad_adjoint(nep_model* m, const nep_system* sys, const nep_nlist* nl,
                                  const double* a_e, const float* lam, const double* mu, float* grad,
                                  void* work, size_t work_bytes, void* stream) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!a_e || !mu || (sys->n_atoms > 0 && !lam)) return fail(NEP_ERR_ARG, "adjoints are NULL");
    if (!grad) return fail(NEP_ERR_ARG, "grad is NULL");
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built");
    if (m->hp.precision != 0)
        return fail(NEP_ERR_UNSUPPORTED, "the gradient is computed for FP32 models (precision 0)");
    if (!m->ks)
        return fail(NEP_ERR_UNSUPPORTED, "no FP32 training operator for this model's shape (generic path): "
                                         "use nep_param_grad_adjoint_fp64");
    TrainLayout tl;
    if ((s = check_train_work(m, sys, nl, work, work_bytes, &tl)) != NEP_OK) return s;
    return train_impl(m, sys, nl, nullptr, nullptr, nullptr, nullptr, 0, a_e, lam, mu, grad, nullptr,
                      work, tl, (cudaStream_t)stream);
}

nep_status nep_adam_step(nep_model* m, const float* grad, float* m1, float* m2, int t, float lr,
                         float beta1, float beta2, float eps, void* stream) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (!grad || !m1 || !m2) return fail(NEP_ERR_ARG, "grad, m1 or m2 is NULL");
    if (t < 1) return fail(NEP_ERR_ARG, "step t must be >= 1");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(NEP_ERR_ARG, "lr must be finite and >= 0");
    if (!(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f))
        return fail(NEP_ERR_ARG, "beta1 and beta2 must lie in [0, 1)");
    if (!(eps > 0.0f) || !std::isfinite(eps)) return fail(NEP_ERR_ARG, "eps must be finite and > 0");
    const int P = (int)nep_num_params(&m->hp);
    const double bc1 = 1.0 - std::pow((double)beta1, (double)t);
    const double bc2 = 1.0 - std::pow((double)beta2, (double)t);
    const float c1 = (float)((double)lr / bc1), c2 = (float)(1.0 / std::sqrt(bc2));
    NEP_CUDA(nep::launch_adam(m->params, grad, m1, m2, P, beta1, beta2, eps, c1, c2, (cudaStream_t)stream),
             "adam");
    return NEP_OK;
}

nep_status nep_selftest_wait_timeout(void* stream) {
    int outcome = 0;
    NEP_CUDA(nep::wait_selftest((cudaStream_t)stream, &outcome), "wait self-test");
    if (outcome & 2) return fail(NEP_ERR_TIMEOUT, "the self-test wait ran out of its poll limit, as designed");
    return NEP_OK;
}

nep_status nep_fp32_peak(void* stream, double* tflops) {
    if (!tflops) return fail(NEP_ERR_ARG, "tflops is NULL");
    NEP_CUDA(nep::fp32_peak((cudaStream_t)stream, tflops), "FP32 peak kernel");
    return NEP_OK;
}

nep_status nep_set_variant(nep_model* m, int size_class, int variant) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (size_class < -1 || size_class >= nep::kSizeBins)
        return fail(NEP_ERR_ARG, "size_class must be -1 or 0..%d", nep::kSizeBins - 1);
    if (variant < -1 || variant >= nep::kVariants)
        return fail(NEP_ERR_ARG, "variant must be -1 or 0..%d", nep::kVariants - 1);
    for (int b = 0; b < nep::kSizeBins; ++b)
        if (size_class < 0 || b == size_class) m->tune_angular[b] = variant;
    return NEP_OK;
}

nep_status nep_set_launch(nep_model* m, int size_class, int variant, int radial_block, int finish_block) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (size_class < -1 || size_class >= nep::kSizeBins)
        return fail(NEP_ERR_ARG, "size_class must be -1 or 0..%d", nep::kSizeBins - 1);
    if (variant < -1 || variant >= nep::kVariants)
        return fail(NEP_ERR_ARG, "variant must be -1 or 0..%d", nep::kVariants - 1);
    if ((radial_block && !block_choice(radial_block)) || (finish_block && !block_choice(finish_block)))
        return fail(NEP_ERR_ARG, "block sizes must be 0 (default), 64, 128 or 256");
    for (int b = 0; b < nep::kSizeBins; ++b)
        if (size_class < 0 || b == size_class) {
            m->tune_angular[b] = variant;
            m->tune_radial[b] = radial_block;
            m->tune_finish[b] = finish_block;
        }
    return NEP_OK;
}

nep_status nep_autotune(nep_model* m, const nep_system* sys, const nep_nlist* nl, void* work,
                        size_t work_bytes, void* stream, int reps, int* chosen) {
    nep_status s;
    if ((s = check_system(m, sys)) != NEP_OK) return s;
    if (!m->ks) return fail(NEP_ERR_UNSUPPORTED, "the generic path has no launch choices to tune");
    if ((s = check_nlist(nl, sys->n_atoms)) != NEP_OK) return s;
    if (!nl->min_image && !nl->shift) return fail(NEP_ERR_STATE, "list was not built");
    if (reps < 1) reps = 1;
    WsLayout w;
    if ((s = check_work(m, sys, nl, work, work_bytes, &w)) != NEP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = sys->n_atoms;
    NEP_CUDA(nep::launch_pack(sys->pos, sys->type, sys->atom_off, N, sys->n_cfg, m->hp.n_types,
                              at<float4>(work, w.pos4), at<int>(work, w.cfg), nl->status, st),
             "pack");
    const nep::EvalArgs a = make_args(m, sys, nl, work, w);
    NEP_CUDA(nep::launch_chunk_plan(sys->atom_off, sys->n_cfg, at<int>(work, w.chunk_start), st), "chunk plan");
    cudaEvent_t e0, e1;
    NEP_CUDA(cudaEventCreate(&e0), "event");
    NEP_CUDA(cudaEventCreate(&e1), "event");
    // one untimed launch, then the best of `reps` timed launches of `launch`
    auto best_of = [&](auto launch, float* tmin) -> cudaError_t {
        *tmin = 1e30f;
        for (int r = 0; r <= reps; ++r) {
            cudaEventRecord(e0, st);
            cudaError_t err = launch();
            cudaEventRecord(e1, st);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err != cudaSuccess) return err;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < *tmin) *tmin = ms;
        }
        return cudaSuccess;
    };
    nep::FinishArgs f;
    f.atom_off = sys->atom_off;
    f.chunk_start = at<int>(work, w.chunk_start);
    f.partial = at<double>(work, w.partial);
    f.force = at<float>(work, w.fpart);   // scratch target: the tuner's forces are not kept
    f.e_out = nullptr;
    f.n_owned = N;
    int vd = nep::kDefaultAngularVariant, rb = 0, fb = 0;
    cudaError_t err = cudaSuccess;
    if (N > 0) {
        // the radial kernel's block size, then the angular variant (on the
        // radial kernel's outputs), then the finish kernel's block size (on
        // the angular kernel's outputs)
        float best = 1e30f, t = 0.0f;
        for (int c : nep::kBlockChoices) {
            if ((err = best_of([&] { return m->ks->radial(a, st, c); }, &t))) break;
            if (t < best) best = t, rb = c;
        }
        best = 1e30f;
        for (int v = 0; v < nep::kVariants && !err; ++v) {
            if ((err = best_of([&] { return m->ks->angular(a, st, v); }, &t))) break;
            if (t < best) best = t, vd = v;
        }
        if (!err) err = m->ks->angular(a, st, vd);
        best = 1e30f;
        for (int c : nep::kBlockChoices) {
            if (err) break;
            if ((err = best_of([&] { return m->ks->finish(a, f, w.max_chunks, st, c); }, &t))) break;
            if (t < best) best = t, fb = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(err, "autotune launch");
    const int b = size_bin(sys);
    m->tune_angular[b] = vd;
    m->tune_radial[b] = rb;
    m->tune_finish[b] = fb;
    if (chosen) {
        chosen[0] = vd;
        chosen[1] = rb;
        chosen[2] = fb;
    }
    return NEP_OK;
}

nep_status nep_set_timing_events(nep_model* m, void* const* events, int n) {
    if (!m) return fail(NEP_ERR_ARG, "model is NULL");
    if (n == 0) {
        m->n_timing = 0;
        return NEP_OK;
    }
    if (n != 4 || !events) return fail(NEP_ERR_ARG, "need exactly 4 events");
    for (int k = 0; k < 4; ++k) {
        if (!events[k]) return fail(NEP_ERR_ARG, "event %d is NULL", k);
        m->timing[k] = (cudaEvent_t)events[k];
    }
    m->n_timing = 4;
    return NEP_OK;
}

nep_status nep_check(const nep_nlist* nl, void* stream) {
    NEP_CUDA(cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
    if (!nl || !nl->status) return NEP_OK;
    int st[4];
    NEP_CUDA(cudaMemcpy(st, nl->status, sizeof st, cudaMemcpyDeviceToHost), "read status");
    if (st[0]) return fail(NEP_ERR_CAPACITY, "neighbour list overflow: need cap >= %d, cap_ang >= %d", st[1], st[2]);
    if (st[3]) return fail(NEP_ERR_INPUT, "invalid input: species out of range, non-finite position or atom outside its box");
    return NEP_OK;
}

}  // extern "C"
