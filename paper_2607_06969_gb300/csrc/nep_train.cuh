// Training backward: gradient of Phi = sum_b aE_b E_b + sum_i lam_i . F_i
// + sum_b mu_b : V_b with respect to every parameter (the loss gradient of
// Eqs. 18-21 when aE, lam, mu are the loss adjoints), without autograd
// caches; per-pair derivatives are recomputed.
//
// With F_i = -dE/dr_i (Eq. 3) and V = -dE/deps (Eq. 4),
//   Phi = sum_k [ aE E_k + sum_j dE_k/dr_kj . dr_kj ],
//   dr_kj = -(lam_j - lam_k) - mu r_kj,
// and sum_j dE_k/dr_kj . dr_kj = p_k . dq_k with p = dE/dq and dq the
// tangent of the descriptors along dr.  Kernels, one thread per atom:
//   tangent : dq (radial via species-resolved sums of Q'_k (rhat . dr),
//             angular via dS_nlm), stored with dS; then, for the same atom,
//             the network second-order terms: alpha, beta, gamma (network
//             gradient coefficients) and rho = aE p + d(p . dq)/dq.
//   xzP/xzR : per angular pair X_n = sum_m P_nm Y_m + sum_m R_nm dY_m . dr and
//             Z_n = (rhat . dr) sum_m R_nm Y_m, where P = dPhi/dS, R = dPhi/d(dS).
//   cbins   : per-atom angular c-gradient sum_j Q_k X_n + Q'_k Z_n by species
//             (X_n = the sum of its P and R planes).
// These four run one after another in one kernel (k_tangent), each thread on
// its own atom; the gradient reduction follows in its own kernels.
//   grad    : per-chunk sums over atoms of every parameter's contributions
//             (tiles of atoms staged in shared memory in species order,
//             accumulators in shared memory), then an FP64 sum over chunks
//             in fixed order.
#pragma once
#include "nep_eval.cuh"
#include "nep_mlp_tc.cuh"

namespace nep {

// resident 128-thread blocks per SM asked of each per-atom training kernel
// (their register budget: 65,536 / (128 x blocks))
#ifndef NEP_MINB_TANGENT
#define NEP_MINB_TANGENT 2
#endif

constexpr int kGradChunk = 32;   // atoms per staged tile
constexpr int kGradTiles = 8;    // most tiles per gradient chunk (one CTA)

NEP_HD int config_of_comp_j(int addr, int N) { return addr - (addr / N) * N; }

NEP_HD void adjoint_frame(const TrainArgs& t, int i, float4& li, float* mu) {
    li = t.lam4[i];
    const int b = t.e.cfg[i];
#pragma unroll
    for (int k = 0; k < 9; ++k) mu[k] = t.mu[9 * b + k];
}

// Pair records of a compacted list read ahead: the record two pairs ahead
// and the neighbour's adjoint one pair ahead, so that the two dependent
// global loads of a pair overlap the work on the pairs before it.  J(e)
// decodes the neighbour index of a record.
template <class J>
struct AdjointStream {
    const float4* rec;     // [slot][N] records of atom i
    const float4* lam4;
    int N, i, n;
    float4 e1, e2, l1;
    J j_of;
    NEP_HD AdjointStream(const float4* rec_, const float4* lam4_, int N_, int i_, int n_, J j)
        : rec(rec_), lam4(lam4_), N(N_), i(i_), n(n_), j_of(j) {
        const float4 z = {0.0f, 0.0f, 0.0f, 0.0f};
        e1 = n > 0 ? rec[i] : z;
        e2 = n > 1 ? rec[N + i] : z;
        l1 = n > 0 ? lam4[j_of(e1)] : z;
    }
    // record and neighbour adjoint of pair c, then the loads for c + 1, c + 2
    NEP_HD void next(int c, float4& e, float4& lj) {
        const float4 z = {0.0f, 0.0f, 0.0f, 0.0f};
        e = e1;
        lj = l1;
        e1 = e2;
        l1 = c + 1 < n ? lam4[j_of(e1)] : z;
        e2 = c + 2 < n ? rec[(size_t)(c + 2) * N + i] : z;
    }
};
struct RadialJ {
    NEP_HD int operator()(float4 e) const { return (int)((unsigned)f2i(e.w) >> 2); }
};
struct AngularJ {
    int N;
    NEP_HD int operator()(float4 e) const { return config_of_comp_j((int)((unsigned)f2i(e.w) >> 2), N); }
};

// dr_ij = -(lam_j - lam_i) - mu r_ij
NEP_HD void pair_tangent(const float* mu, float4 li, float4 lj, float rx, float ry, float rz,
                         float& dx, float& dy, float& dz) {
    dx = -(lj.x - li.x) - (mu[0] * rx + mu[1] * ry + mu[2] * rz);
    dy = -(lj.y - li.y) - (mu[3] * rx + mu[4] * ry + mu[5] * rz);
    dz = -(lj.z - li.z) - (mu[6] * rx + mu[7] * ry + mu[8] * rz);
}

// ---------------------------------------------------------------------------
template <class C>
NEP_HD void tangent_atom(const TrainArgs& t, const float* sm, int i) {
    constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T, D = C::D;
    const EvalArgs& a = t.e;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N;
    const int ti = f2i(a.pos4[i].w);
    const float irR = 1.0f / a.rc_rad, irA = 1.0f / a.rc_ang;
    float4 li;
    float mu[9];
    adjoint_frame(t, i, li, mu);

    // radial: DF[t][k] = sum_{j of species t} Q'_k(r) (rhat . dr)
    float df[T][KR];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int k = 0; k < KR; ++k) df[s][k] = 0.0f;
    const int ncr = a.cnt_compr[i];
    AdjointStream<RadialJ> rs(a.compr, t.lam4, N, i, ncr, RadialJ{});
    for (int s = 0; s < ncr; ++s) {
        float4 e, lj;
        rs.next(s, e, lj);
        const int tj = f2i(e.w) & 3;
        float drx, dry, drz;
        pair_tangent(mu, li, lj, e.x, e.y, e.z, drx, dry, drz);
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        const float ir = rcp_f(r);
        const float udr = (e.x * drx + e.y * dry + e.z * drz) * ir;
        float f[KR], fp[KR];
        basis_d<KR>(r, irR, f, fp);
#pragma unroll
        for (int s2 = 0; s2 < T; ++s2) {
            const float w = (tj == s2) ? udr : 0.0f;
#pragma unroll
            for (int k = 0; k < KR; ++k) df[s2][k] = fmaf(w, fp[k], df[s2][k]);
        }
    }
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int k = 0; k < KR; ++k) t.df[(s * KR + k) * N + i] = df[s][k];
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int s = 0; s < T; ++s) {
            const float* c = sm + sl.cR + (ti * T + s) * C::SR + n * KR;
#pragma unroll
            for (int k = 0; k < KR; ++k) acc = fmaf(c[k], df[s][k], acc);
        }
        t.dq[n * N + i] = acc;
        NEP_SCHED_BARRIER();
    }

    // angular: dS_nlm = sum_j [g'_n (rhat.dr) Y_m + g_n (grad P_m . dr - l Y_m rhat.dr)/r]
    float dS[NA][kLM];
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int m = 0; m < kLM; ++m) dS[n][m] = 0.0f;
    const int nc = a.cnt_comp[i];
    AdjointStream<AngularJ> as(a.comp, t.lam4, N, i, nc, AngularJ{N});
    for (int c = 0; c < nc; ++c) {
        float4 e, lj;
        as.next(c, e, lj);
        const int tj = f2i(e.w) & 3;
        float drx, dry, drz;
        pair_tangent(mu, li, lj, e.x, e.y, e.z, drx, dry, drz);
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        const float ir = rcp_f(r);
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        const float udr = ht.x * drx + ht.y * dry + ht.z * drz;
        float g[NA], gp[NA];
        {
            float f[KA], fp[KA];
            basis_d<KA>(r, irA, f, fp);
            const float* cc = sm + sl.cA + (ti * T + tj) * C::SA;
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                float u = 0.0f, v = 0.0f;
#pragma unroll
                for (int k = 0; k < KA; ++k) {
                    u = fmaf(cc[n * KA + k], f[k], u);
                    v = fmaf(cc[n * KA + k], fp[k], v);
                }
                g[n] = u;
                gp[n] = v;
            }
        }
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            float Y, hx, hy, hz;
            harm_m(m, ht, Y, hx, hy, hz);
            const float gdr = (hx * drx + hy * dry + hz * drz) * ir;
            const float yu = Y * udr;
            const float lr = (float)lm_l(m) * ir;
#pragma unroll
            for (int n = 0; n < NA; ++n)
                dS[n][m] = fmaf(yu, fmaf(-lr, g[n], gp[n]), fmaf(g[n], gdr, dS[n][m]));
        }
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float S[kLM];
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            S[m] = a.S[(n * kLM + m) * N + i];
            t.dS[(n * kLM + m) * N + i] = dS[n][m];
        }
        float dql[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int m = 0; m < kLM; ++m) dql[lm_l(m) - 1] = fmaf(2.0f * clm(m) * S[m], dS[n][m], dql[lm_l(m) - 1]);
#pragma unroll
        for (int l = 0; l < 4; ++l) t.dq[(NR + n * 4 + l) * N + i] = dql[l];
        if (C::H4) {
            float J[5], S2[5] = {S[3], S[4], S[5], S[6], S[7]};
            fourbody(S2, J);
            float v = 0.0f;
#pragma unroll
            for (int m = 0; m < 5; ++m) v = fmaf(J[m], dS[n][3 + m], v);
            t.dq[(NR + NA * 4 + n) * N + i] = v;
        }
        NEP_SCHED_BARRIER();
    }
    (void)D;
}

// ---------------------------------------------------------------------------
template <class C>
NEP_HD void mlp2_atom(const TrainArgs& t, const float* sm, int i) {
    constexpr int D = C::D;
    const EvalArgs& a = t.e;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N, H = a.H;
    const int ti = f2i(a.pos4[i].w);
    const float aE = t.aE[a.cfg[i]];
    const float* W0 = sm + sl.W0 + ti * sl.SW;
    const float* b0 = sm + sl.b0 + ti * sl.HS;
    const float* w1 = sm + sl.w1 + ti * sl.HS;
    float q[D], dq[D], p2[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        q[d] = a.q_out[d * N + i];
        dq[d] = t.dq[d * N + i];
        p2[d] = 0.0f;
    }
    for (int h = 0; h < H; ++h) {
        const float* w = W0 + h * C::DW;
        float z = b0[h], u = 0.0f;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            z = fmaf(w[d], q[d], z);
            u = fmaf(w[d], dq[d], u);
        }
        const float th = tanh_f(z);
        const float s = 1.0f - th * th;
        const float wh = w1[h];
        const float c2 = -2.0f * wh * u * th * s;     // d(w1 s u)/dz
        t.coef[h * N + i] = aE * wh * s + c2;          // alpha: coefficient of q in dW0, and db0
        t.coef[(H + h) * N + i] = wh * s;              // beta: coefficient of dq in dW0
        t.coef[(2 * H + h) * N + i] = aE * th + s * u; // gamma: dw1
#pragma unroll
        for (int d = 0; d < D; ++d) p2[d] = fmaf(c2, w[d], p2[d]);
    }
#pragma unroll
    for (int d = 0; d < D; ++d) t.rho[d * N + i] = fmaf(aE, a.p_out[d * N + i], p2[d]);
}

// ---------------------------------------------------------------------------
// X_n from P = dPhi/dS (pass 1)
template <class C>
NEP_HD void xzp_atom(const TrainArgs& t, const float* sm, int i) {
    constexpr int NR = C::NR, NA = C::NA;
    const EvalArgs& a = t.e;
    const int N = a.N, capA = a.cap_ang;
    float P[NA][kLM];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float rl[4], pl[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            rl[l] = t.rho[(NR + n * 4 + l) * N + i];
            pl[l] = a.p_out[(NR + n * 4 + l) * N + i];
        }
        float S2[5], dS2[5];
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            const float S = a.S[(n * kLM + m) * N + i];
            const float dS = t.dS[(n * kLM + m) * N + i];
            if (m >= 3 && m < 8) { S2[m - 3] = S; dS2[m - 3] = dS; }
            P[n][m] = 2.0f * clm(m) * fmaf(rl[lm_l(m) - 1], S, pl[lm_l(m) - 1] * dS);
        }
        if (C::H4) {
            const float r4 = t.rho[(NR + NA * 4 + n) * N + i];
            const float p4 = a.p_out[(NR + NA * 4 + n) * N + i];
            float J[5], dJ[5];
            fourbody_jvp(S2, dS2, J, dJ);
#pragma unroll
            for (int m = 0; m < 5; ++m) P[n][3 + m] = fmaf(r4, J[m], fmaf(p4, dJ[m], P[n][3 + m]));
        }
    }
    const int nc = a.cnt_comp[i];
    for (int c = 0; c < nc; ++c) {
        const float4 e = a.comp[c * N + i];
        const float ir = rcp_f(sqrt_f(dist2(e.x, e.y, e.z)));
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        float X[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) X[n] = 0.0f;
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            float Y, hx, hy, hz;
            harm_m(m, ht, Y, hx, hy, hz);
#pragma unroll
            for (int n = 0; n < NA; ++n) X[n] = fmaf(P[n][m], Y, X[n]);
        }
#pragma unroll
        for (int n = 0; n < NA; ++n) t.xz[((size_t)n * capA + c) * N + i] = X[n];
    }
}

// X_n's second part sum_m R dY_m . dr and Z_n = (rhat.dr) sum_m R Y_m with
// R = dPhi/d(dS) (pass 2); the two parts of X_n sit in separate planes, so
// this pass only writes
template <class C>
NEP_HD void xzr_atom(const TrainArgs& t, const float* sm, int i) {
    constexpr int NR = C::NR, NA = C::NA;
    (void)sm;
    const EvalArgs& a = t.e;
    const int N = a.N, capA = a.cap_ang;
    float R[NA][kLM];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float pl[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) pl[l] = a.p_out[(NR + n * 4 + l) * N + i];
        float S2[5];
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            const float S = a.S[(n * kLM + m) * N + i];
            if (m >= 3 && m < 8) S2[m - 3] = S;
            R[n][m] = 2.0f * clm(m) * pl[lm_l(m) - 1] * S;
        }
        if (C::H4) {
            const float p4 = a.p_out[(NR + NA * 4 + n) * N + i];
            float J[5];
            fourbody(S2, J);
#pragma unroll
            for (int m = 0; m < 5; ++m) R[n][3 + m] = fmaf(p4, J[m], R[n][3 + m]);
        }
    }
    float4 li;
    float mu[9];
    adjoint_frame(t, i, li, mu);
    const int nc = a.cnt_comp[i];
    AdjointStream<AngularJ> as(a.comp, t.lam4, N, i, nc, AngularJ{N});
    for (int c = 0; c < nc; ++c) {
        float4 e, lj;
        as.next(c, e, lj);
        float drx, dry, drz;
        pair_tangent(mu, li, lj, e.x, e.y, e.z, drx, dry, drz);
        const float ir = rcp_f(sqrt_f(dist2(e.x, e.y, e.z)));
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        const float udr = ht.x * drx + ht.y * dry + ht.z * drz;
        float X[NA], Z[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            X[n] = 0.0f;
            Z[n] = 0.0f;
        }
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            float Y, hx, hy, hz;
            harm_m(m, ht, Y, hx, hy, hz);
            const float dY = ((hx * drx + hy * dry + hz * drz) - (float)lm_l(m) * Y * udr) * ir;
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                X[n] = fmaf(R[n][m], dY, X[n]);
                Z[n] = fmaf(R[n][m], Y, Z[n]);
            }
        }
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            t.xz[((size_t)(2 * NA + n) * capA + c) * N + i] = X[n];
            t.xz[((size_t)(NA + n) * capA + c) * N + i] = udr * Z[n];
        }
    }
}

// per-atom angular c-gradient: bins[t][n][k] = sum_{j of species t} Q_k X_n + Q'_k Z_n
template <class C>
NEP_HD void cbins_atom(const TrainArgs& t, const float* sm, int i) {
    constexpr int NA = C::NA, KA = C::KA, T = C::T;
    (void)sm;
    const EvalArgs& a = t.e;
    const int N = a.N, capA = a.cap_ang;
    const float irA = 1.0f / a.rc_ang;
    float bins[T][NA][KA];
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int n = 0; n < NA; ++n)
#pragma unroll
            for (int k = 0; k < KA; ++k) bins[s][n][k] = 0.0f;
    const int nc = a.cnt_comp[i];
    for (int c = 0; c < nc; ++c) {
        const float4 e = a.comp[c * N + i];
        const int tj = f2i(e.w) & 3;
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        float f[KA], fp[KA];
        basis_d<KA>(r, irA, f, fp);
        float X[NA], Z[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            X[n] = t.xz[((size_t)n * capA + c) * N + i] + t.xz[((size_t)(2 * NA + n) * capA + c) * N + i];
            Z[n] = t.xz[((size_t)(NA + n) * capA + c) * N + i];
        }
#pragma unroll
        for (int s = 0; s < T; ++s) {
            if (tj == s) {
#pragma unroll
                for (int n = 0; n < NA; ++n)
#pragma unroll
                    for (int k = 0; k < KA; ++k) bins[s][n][k] = fmaf(f[k], X[n], fmaf(fp[k], Z[n], bins[s][n][k]));
            }
        }
    }
#pragma unroll
    for (int s = 0; s < T; ++s)
#pragma unroll
        for (int n = 0; n < NA; ++n)
#pragma unroll
            for (int k = 0; k < KA; ++k) t.bins[((s * NA + n) * KA + k) * N + i] = bins[s][n][k];
}

// ---------------------------------------------------------------------------
// Gradient partials: every parameter's contribution summed over a staged
// tile of kGradChunk atoms whose rows are in species order.
//
// A staged row holds, per atom (floats): the species bits and dE_b/dE of its
// configuration, then q and dq, alpha, beta and gamma, rho and p (radial n),
// the species-resolved basis sums F and DF (one block of K_R per species),
// and the angular c-gradient bins.  Every block starts on a multiple of 4
// (16 bytes) and is padded to a multiple of 4, so that four consecutive
// entries are one vector load.  The logical field order (the staging
// sources) is the same without the padding.
template <class C>
struct GradStage {
    static constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T, D = C::D;
    static constexpr int Dp = (D + 3) & ~3, NRp = (NR + 3) & ~3, KRp = (KR + 3) & ~3;
    static constexpr int NBINS = T * NA * KA, NBp = (NBINS + 3) & ~3;
    static NEP_HD int Hp(int H) { return (H + 3) & ~3; }
    static NEP_HD int o_q() { return 4; }
    static NEP_HD int o_dq() { return 4 + Dp; }
    static NEP_HD int o_al() { return 4 + 2 * Dp; }
    static NEP_HD int o_be(int H) { return o_al() + Hp(H); }
    static NEP_HD int o_ga(int H) { return o_be(H) + Hp(H); }
    static NEP_HD int o_rho(int H) { return o_ga(H) + Hp(H); }
    static NEP_HD int o_p(int H) { return o_rho(H) + NRp; }
    static NEP_HD int o_fb(int H) { return o_p(H) + NRp; }
    static NEP_HD int o_df(int H) { return o_fb(H) + T * KRp; }
    static NEP_HD int o_bins(int H) { return o_df(H) + T * KRp; }
    // row stride: a multiple of 4 (16-byte rows) with W/4 odd, so that 8
    // consecutive rows start in 8 distinct groups of 4 banks
    static NEP_HD int width(int H) {
        const int w = o_bins(H) + NBp;
        return (w & 4) ? w : w + 4;
    }
    // logical fields: 2 + 2D + 3H + 2 NR + 2 T KR + T NA KA
    static NEP_HD int fields(int H) { return 2 + 2 * D + 3 * H + 2 * NR + 2 * T * KR + NBINS; }
    // column of logical field f in the padded row
    static NEP_HD int column(int f, int H) {
        if (f < 2) return f;
        f -= 2;
        if (f < D) return o_q() + f;
        f -= D;
        if (f < D) return o_dq() + f;
        f -= D;
        if (f < 3 * H) return o_al() + (f / H) * Hp(H) + f % H;
        f -= 3 * H;
        if (f < NR) return o_rho(H) + f;
        f -= NR;
        if (f < NR) return o_p(H) + f;
        f -= NR;
        if (f < T * KR) return o_fb(H) + (f / KR) * KRp + f % KR;
        f -= T * KR;
        if (f < T * KR) return o_df(H) + (f / KR) * KRp + f % KR;
        f -= T * KR;
        return o_bins(H) + f;
    }
};

// address of logical field f of atom i
template <class C>
NEP_HD const float* stage_src(const TrainArgs& t, int f, int i) {
    constexpr int NR = C::NR, KR = C::KR, T = C::T, D = C::D;
    const EvalArgs& a = t.e;
    const size_t N = a.N;
    const int H = a.H;
    if (f == 0) return &a.pos4[i].w;
    if (f == 1) return t.aE + a.cfg[i];
    f -= 2;
    if (f < D) return a.q_out + f * N + i;
    f -= D;
    if (f < D) return t.dq + f * N + i;
    f -= D;
    if (f < 3 * H) return t.coef + f * N + i;
    f -= 3 * H;
    if (f < NR) return t.rho + f * N + i;
    f -= NR;
    if (f < NR) return a.p_out + f * N + i;
    f -= NR;
    if (f < T * KR) return a.fb_out + f * N + i;
    f -= T * KR;
    if (f < T * KR) return t.df + f * N + i;
    f -= T * KR;
    return t.bins + f * N + i;
}

// tiles of kGradChunk atoms per gradient chunk: enough chunks to fill the
// GPU (about 512), at most kGradTiles; a function of N alone, so that the
// summation order does not depend on the device
NEP_HD int grad_tiles_per_chunk(int N) {
    const int tiles = (N + kGradChunk - 1) / kGradChunk;
    const int k = (tiles + 511) / 512;
    return k < 1 ? 1 : (k > kGradTiles ? kGradTiles : k);
}
NEP_HD int grad_chunks_of(int N) {
    const int per = kGradChunk * grad_tiles_per_chunk(N);
    return (N + per - 1) / per;
}

// Work items of a tile: each sums, over the staged rows of its species,
// four parameters of one block that read four consecutive columns, or for
// W0 a 4 x 4 block of them (per atom four 16-byte loads for 32 FMAs):
//   W0  (species, h0..h0+3, d0..d0+3):  alpha_h q_d + beta_h dq_d
//   b0  (species, h0..h0+3):       alpha_h
//   w1  (species, h0..h0+3):       gamma_h
//   b1  (species):                 dPhi/dE of the atom's configuration
//   cR  (t1, t2, n, k0..k0+3):     rho_n F[t2][k] + p_n DF[t2][k]
//   cA  (t1, bins b0..b0+3):       bins[b]
template <class C>
struct GradItems {
    using G = GradStage<C>;
    static constexpr int T = C::T;
    static NEP_HD int nW0(int H) { return T * (G::Hp(H) / 4) * (G::Dp / 4); }
    static NEP_HD int nB(int H) { return T * (G::Hp(H) / 4); }
    static constexpr int nCR = T * T * C::NR * (G::KRp / 4);
    static constexpr int nCA = T * (G::NBp / 4);
    static NEP_HD int total(int H) { return nW0(H) + 2 * nB(H) + T + nCR + nCA; }
};

template <class C>
NEP_HD void grad_item(const float* stage, const int* toff, int H, int it, float* acc) {
    using G = GradStage<C>;
    using I = GradItems<C>;
    constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T, D = C::D;
    const int W = G::width(H);
    const ParamLayout L = param_layout(T, NR, NA, KR, KA, C::H4, H);
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    int sp, pbase, cnt;
    if (it < I::nW0(H)) {
        // each parameter's chain is the same as with one h per item: the
        // same operations over the same atoms in the same order
        constexpr int NB = G::Dp / 4;
        const int HB = G::Hp(H) / 4;
        sp = it / (HB * NB);
        const int rem = it % (HB * NB), h0 = 4 * (rem / NB), d0 = 4 * (rem % NB);
        float acc4[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc4[r][c] = 0.0f;
        for (int a = toff[sp]; a < toff[sp + 1]; ++a) {
            const float* row = stage + a * W;
            const float4 al4 = *reinterpret_cast<const float4*>(row + G::o_al() + h0);
            const float4 be4 = *reinterpret_cast<const float4*>(row + G::o_be(H) + h0);
            const float4 q4 = *reinterpret_cast<const float4*>(row + G::o_q() + d0);
            const float4 dq4 = *reinterpret_cast<const float4*>(row + G::o_dq() + d0);
            const float al[4] = {al4.x, al4.y, al4.z, al4.w}, be[4] = {be4.x, be4.y, be4.z, be4.w};
            const float q[4] = {q4.x, q4.y, q4.z, q4.w}, dq[4] = {dq4.x, dq4.y, dq4.z, dq4.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc4[r][c] = fmaf(be[r], dq[c], fmaf(al[r], q[c], acc4[r][c]));
        }
        // rows h >= H and columns d >= D are padding: their sums are dropped
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (h0 + r >= H) break;
            const int pb = sp * L.mlp_stride + (h0 + r) * D + d0;
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (d0 + c < D) acc[pb + c] += acc4[r][c];
        }
        return;
    } else if ((it -= I::nW0(H)) < 2 * I::nB(H)) {
        const int which = it / I::nB(H), r = it % I::nB(H), HB = G::Hp(H) / 4;
        sp = r / HB;
        const int h0 = 4 * (r % HB);
        const int col = (which ? G::o_ga(H) : G::o_al()) + h0;
        for (int a = toff[sp]; a < toff[sp + 1]; ++a) {
            const float4 v = *reinterpret_cast<const float4*>(stage + a * W + col);
            s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
        }
        pbase = sp * L.mlp_stride + H * D + which * H + h0;
        cnt = H - h0;
    } else if ((it -= 2 * I::nB(H)) < T) {
        sp = it;
        for (int a = toff[sp]; a < toff[sp + 1]; ++a) s0 += stage[a * W + 1];
        pbase = sp * L.mlp_stride + H * D + 2 * H;
        cnt = 1;
    } else if ((it -= T) < I::nCR) {
        constexpr int KB = G::KRp / 4;
        const int k0 = 4 * (it % KB);
        int x = it / KB;
        const int n = x % NR;
        x /= NR;
        const int t2 = x % T;
        sp = x / T;
        for (int a = toff[sp]; a < toff[sp + 1]; ++a) {
            const float* row = stage + a * W;
            const float rho = row[G::o_rho(H) + n], pn = row[G::o_p(H) + n];
            const float4 F = *reinterpret_cast<const float4*>(row + G::o_fb(H) + t2 * G::KRp + k0);
            const float4 DF = *reinterpret_cast<const float4*>(row + G::o_df(H) + t2 * G::KRp + k0);
            s0 = fmaf(pn, DF.x, fmaf(rho, F.x, s0));
            s1 = fmaf(pn, DF.y, fmaf(rho, F.y, s1));
            s2 = fmaf(pn, DF.z, fmaf(rho, F.z, s2));
            s3 = fmaf(pn, DF.w, fmaf(rho, F.w, s3));
        }
        pbase = L.off_cR + ((sp * T + t2) * NR + n) * KR + k0;
        cnt = KR - k0;
    } else {
        it -= I::nCR;
        constexpr int BB = G::NBp / 4;
        sp = it / BB;
        const int b0 = 4 * (it % BB);
        for (int a = toff[sp]; a < toff[sp + 1]; ++a) {
            const float4 v = *reinterpret_cast<const float4*>(stage + a * W + G::o_bins(H) + b0);
            s0 += v.x; s1 += v.y; s2 += v.z; s3 += v.w;
        }
        pbase = L.off_cA + sp * G::NBINS + b0;
        cnt = G::NBINS - b0;
    }
    acc[pbase] += s0;
    if (cnt > 1) acc[pbase + 1] += s1;
    if (cnt > 2) acc[pbase + 2] += s2;
    if (cnt > 3) acc[pbase + 3] += s3;
}

#if defined(__CUDACC__)
// The per-atom backward of one atom in one thread: the tangent pass, the
// network's second-order terms, the X and Z coefficients of its angular
// pairs (P and R passes) and its angular c-gradient bins.  Each step needs
// only this atom's own results of the steps before it (and inputs), so the
// passes run back to back with no launch between them.
template <class C>
__global__ void __launch_bounds__(kBlock, NEP_MINB_TANGENT) k_tangent(const TrainArgs t) {
    extern __shared__ float sm[];
    load_model<C>(sm, t.e.params, t.e.H, threadIdx.x, blockDim.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < t.e.N) {
        tangent_atom<C>(t, sm, i);
        mlp2_atom<C>(t, sm, i);
        xzp_atom<C>(t, nullptr, i);
        xzr_atom<C>(t, nullptr, i);
        cbins_atom<C>(t, nullptr, i);
    }
}
constexpr int kGradThreads = 256;
constexpr int kStageUnroll = 8;
// shared memory of k_grad_partial: the staged tile, the field tables, the
// chunk's accumulators
template <class C>
struct GradSmem {
    size_t stage, src, col, acc, total;   // byte offsets
};
template <class C>
NEP_HD GradSmem<C> grad_smem(int H) {
    using G = GradStage<C>;
    const ParamLayout L = param_layout(C::T, C::NR, C::NA, C::KR, C::KA, C::H4, H);
    GradSmem<C> m;
    m.stage = 0;
    m.src = m.stage + sizeof(float) * (size_t)kGradChunk * G::width(H);        // 16-byte multiple
    m.col = m.src + sizeof(const float*) * (size_t)G::fields(H);
    m.acc = m.col + sizeof(int) * (size_t)G::fields(H);
    m.total = m.acc + sizeof(float) * (size_t)L.P;
    return m;
}

// one chunk of grad_tiles_per_chunk(N) tiles of kGradChunk atoms per CTA:
// each tile is staged in shared memory with its rows in species order
// (stable), every thread adds its work items' sums over the tile to shared
// accumulators, and the chunk's partials go out once
template <class C>
__global__ void __launch_bounds__(kGradThreads) k_grad_partial(const TrainArgs t) {
    using G = GradStage<C>;
    constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T;
    extern __shared__ float4 smem4[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(smem4);
    __shared__ int toff[T + 1];
    __shared__ int rowatom[kGradChunk];
    const EvalArgs& a = t.e;
    const int H = a.H, N = a.N;
    const int W = G::width(H), WF = G::fields(H);
    const ParamLayout L = param_layout(T, NR, NA, KR, KA, C::H4, H);
    const GradSmem<C> sm = grad_smem<C>(H);
    float* stage = reinterpret_cast<float*>(smem + sm.stage);        // [kGradChunk][W]
    const float** src = reinterpret_cast<const float**>(smem + sm.src);  // [WF] field bases
    int* col = reinterpret_cast<int*>(smem + sm.col);                // [WF] field columns
    float* acc = reinterpret_cast<float*>(smem + sm.acc);            // [P]
    for (int p = threadIdx.x; p < L.P; p += blockDim.x) acc[p] = 0.0f;
    for (int f = threadIdx.x; f < WF; f += blockDim.x) {
        src[f] = f >= 2 ? stage_src<C>(t, f, 0) : nullptr;
        col[f] = G::column(f, H);
    }
    const int NI = GradItems<C>::total(H);
    const int tpc = grad_tiles_per_chunk(N);
    const int c0 = blockIdx.x * tpc * kGradChunk;
    for (int tile = 0; tile < tpc; ++tile) {
        const int a0 = c0 + tile * kGradChunk;
        if (a0 >= N) break;
        const int na = min(kGradChunk, N - a0);
        // rows in species order: warp 0, one lane per atom
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int sp = lane < na ? f2i(a.pos4[a0 + lane].w) : T;
            int base = 0, pos = 0;
            for (int s2 = 0; s2 <= T; ++s2) {
                const unsigned m = __ballot_sync(0xffffffffu, sp == s2);
                if (s2 < T && lane == 0) toff[s2] = base;
                if (sp == s2) pos = base + __popc(m & ((1u << lane) - 1u));
                base += __popc(m);
            }
            if (lane == 0) toff[T] = na;
            if (lane < na) rowatom[pos] = lane;
        }
        __syncthreads();
        // staging in patches of 8 rows x 4 fields per warp: the 8 rows' atoms
        // lie in the tile's 128-byte window of each field, and the stores of
        // a patch fall in 32 distinct banks; kStageUnroll loads in flight per
        // thread before the stores
        const int total = (kGradChunk / 8) * ((WF + 3) / 4) * 32;
        for (int x0 = threadIdx.x; x0 < total; x0 += kStageUnroll * kGradThreads) {
            float v[kStageUnroll];
#pragma unroll
            for (int u = 0; u < kStageUnroll; ++u) {
                const int x = x0 + u * kGradThreads;
                const int w = x >> 5, l = x & 31;
                const int k = (w % (kGradChunk / 8)) * 8 + (l & 7), f = (w / (kGradChunk / 8)) * 4 + (l >> 3);
                const bool ok = x < total && f < WF && k < na;
                const int fv = ok ? f : 2;
                const int i = a0 + (ok ? rowatom[k] : 0);
                const float* p = fv >= 2 ? src[fv] + i : (fv == 0 ? &a.pos4[i].w : t.aE + a.cfg[i]);
                v[u] = __ldg(p);
            }
#pragma unroll
            for (int u = 0; u < kStageUnroll; ++u) {
                const int x = x0 + u * kGradThreads;
                const int w = x >> 5, l = x & 31;
                const int k = (w % (kGradChunk / 8)) * 8 + (l & 7), f = (w / (kGradChunk / 8)) * 4 + (l >> 3);
                if (x < total && f < WF && k < na) stage[k * W + col[f]] = v[u];
            }
        }
        __syncthreads();
        for (int it = threadIdx.x; it < NI; it += blockDim.x) grad_item<C>(stage, toff, H, it, acc);
        __syncthreads();
    }
    for (int p = threadIdx.x; p < L.P; p += blockDim.x) t.gpart[(size_t)blockIdx.x * L.P + p] = acc[p];
}
// FP64 sum over chunks: 32 parameters per CTA, 8 groups of chunks
// (k = g mod 8) summed in order, then the 8 group sums in order
constexpr int kFinalGroups = 8;
template <class C>
__global__ void __launch_bounds__(32 * kFinalGroups) k_grad_final(const TrainArgs t, int nchunk) {
    __shared__ double part[kFinalGroups][32];
    const ParamLayout L = param_layout(C::T, C::NR, C::NA, C::KR, C::KA, C::H4, t.e.H);
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int p = blockIdx.x * 32 + lane;
    double acc = 0.0;
    if (p < L.P)
        for (int k = g; k < nchunk; k += kFinalGroups) acc += (double)t.gpart[(size_t)k * L.P + p];
    part[g][lane] = acc;
    __syncthreads();
    if (g == 0 && p < L.P) {
        double s = 0.0;
        for (int q = 0; q < kFinalGroups; ++q) s += part[q][lane];
        t.grad[p] = (float)s;
    }
}

template <class C>
size_t grad_stage_bytes(int H) { return grad_smem<C>(H).total; }

// attributes of the training kernels and of the tensor-core network
template <class C>
cudaError_t train_init_t(int H) {
    const int smem = (int)smem_bytes_of<C>(H);
    cudaError_t e;
    if ((e = mlp_tc_init_t<C>(H))) return e;
    if ((e = cudaFuncSetAttribute(k_tangent<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    return cudaFuncSetAttribute(k_grad_partial<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)grad_stage_bytes<C>(H));
}

template <class C>
int grad_chunks_t(int N) { return grad_chunks_of(N); }

template <class C>
cudaError_t train_t(const TrainArgs& t, cudaStream_t st) {
    const int N = t.e.N;
    const size_t smem = smem_bytes_of<C>(t.e.H);
    if (N > 0) {
        const int grid = (N + kBlock - 1) / kBlock;
        k_tangent<C><<<grid, kBlock, smem, st>>>(t);
        k_grad_partial<C><<<grad_chunks_t<C>(N), kGradThreads, grad_stage_bytes<C>(t.e.H), st>>>(t);
    }
    const ParamLayout L = param_layout(C::T, C::NR, C::NA, C::KR, C::KA, C::H4, t.e.H);
    k_grad_final<C><<<(L.P + 31) / 32, 32 * kFinalGroups, 0, st>>>(t, grad_chunks_t<C>(N));
    return cudaGetLastError();
}
#endif

}  // namespace nep
