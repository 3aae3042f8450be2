// Per-atom NEP kernels, templated on the compiled hyper-parameters.  One
// thread owns one atom i in each of them, so every sum over neighbours is a
// private register sum (no atomics, bitwise reproducible).
//
//   k_radial   radial descriptor sums over the neighbour list (Eqs. 11-15),
//              resolved by neighbour species, and compaction of the pairs
//              inside the angular cutoff.  Few registers: many resident warps
//              hide the neighbour gathers.
//   k_angular  angular S_nlm (Eq. 16) over the compacted pairs, q_nl (Eq. 17)
//              and the 4-body term, the per-species tanh network (Section 2.3)
//              and dE/dq, then dE/dS and the angular pair forces f_ij =
//              dE_i/dr_ij, scattered to the reverse slot of the pair.  S and
//              dE/dS stay on the SM.
//   k_finish   radial pair forces of both directions of every pair from the
//              species-projected adjoints, plus the scattered angular forces,
//              give F_i (Eq. 3); per-atom virials (Eq. 4) and energies are
//              summed per chunk of atoms in a fixed order (two-sum FP32 pairs
//              inside a warp, FP64 across warps and chunks).
// In mixed precision k_angular_tc (nep_mlp_tc.cuh) takes k_angular's place
// with the network on the tensor cores.
#pragma once
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nep_device.cuh"
#include "nep_tmem.cuh"

namespace nep {

// Keeps the compiler from hoisting every shared-memory load of a fully
// unrolled contraction ahead of its FMAs (which costs registers and spills).
#if defined(__CUDA_ARCH__)
#define NEP_SCHED_BARRIER() asm volatile("" ::: "memory")
#else
#define NEP_SCHED_BARRIER() ((void)0)
#endif

// Shared-memory row strides: multiples of 4 floats (16-byte vector loads)
// congruent to 4 mod 32, so that the up to 9 species pairs (or 3 species) a
// warp meets land in different 4-bank groups.
NEP_HD constexpr int stride4(int x) { return (x + 31) / 32 * 32 + 4; }
NEP_HD constexpr int round4(int x) { return (x + 3) / 4 * 4; }

NEP_HD float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }

template <int NR_, int NA_, int KR_, int KA_, int H4_, int T_>
struct Cfg {
    static constexpr int NR = NR_, NA = NA_, KR = KR_, KA = KA_, H4 = H4_, T = T_;
    static constexpr int D = NR + NA * 4 + (H4 ? NA : 0);
    static constexpr int NP = NA * (4 + (H4 ? 1 : 0));   // angular + 4-body descriptor count
    static constexpr int SA = stride4(NA * KA);          // per-species-pair stride
    static_assert((NA + NA % 2) * KA <= SA, "the row-paired angular block fits the stride");
    static constexpr int SR = stride4(NR * KR);
    static constexpr int DW = round4(D);                  // row stride of W0 (zero padded)
};

// Shared-memory image of the model, padded so that the (up to 9) species
// pairs or 3 species met by one warp fall in distinct banks.
struct SmemLayout {
    int cA, cA2, cR, W0, b0, w1, b1, total;
    int SW, HS;
};

template <class C>
NEP_HD SmemLayout smem_layout(int H) {
    SmemLayout s;
    s.SW = stride4(H * C::DW);
    s.HS = (H % 2) ? H : H + 1;
    s.cA = 0;
    s.cA2 = s.cA + C::T * C::T * C::SA;   // cA again, rows paired: (c[2p][k], c[2p+1][k])
    s.cR = s.cA2 + C::T * C::T * C::SA;
    s.W0 = s.cR + C::T * C::T * C::SR;
    s.b0 = s.W0 + C::T * s.SW;
    s.w1 = s.b0 + C::T * s.HS;
    s.b1 = s.w1 + C::T * s.HS;
    s.total = s.b1 + C::T;
    return s;
}

// Position of c[n][k] in a row-paired coefficient block: rows 2p and 2p+1
// interleaved, (c[2p][k], c[2p+1][k]) at 2 (p K + k); an odd last row pairs
// with zeros.
template <int K>
NEP_HD int pair_index(int n, int k) { return 2 * ((n / 2) * K + k) + (n % 2); }

// g[n] = sum_k c[n][k] f[k] for n < NA from a row-paired block c2, two rows
// per paired FMA: each g[n] is the same chain, in the same k order, as a
// scalar loop over its row
template <int NA, int K>
NEP_HD void contract_pairs(const float* c2, const float* f, float* g) {
    float2 fb[K];
#pragma unroll
    for (int k = 0; k < K; ++k) fb[k] = make_float2(f[k], f[k]);
#pragma unroll
    for (int p = 0; p < (NA + 1) / 2; ++p) {
        float2 acc = make_float2(0.0f, 0.0f);
        const float* row = c2 + 2 * p * K;
        if (K % 2 == 0) {
#pragma unroll
            for (int k = 0; k < K; k += 2) {
                const float4 v = ld4(row + 2 * k);
                acc = ffma2(make_float2(v.x, v.y), fb[k], acc);
                acc = ffma2(make_float2(v.z, v.w), fb[k + 1], acc);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) acc = ffma2(*reinterpret_cast<const float2*>(row + 2 * k), fb[k], acc);
        }
        g[2 * p] = acc.x;
        if (2 * p + 1 < NA) g[2 * p + 1] = acc.y;
    }
}

// Fill the padded model image from the flat parameter vector; thread `tid`
// of `nthr` copies its share.
template <class C>
NEP_HD void load_model(float* sm, const float* prm, int H, int tid, int nthr) {
    const SmemLayout s = smem_layout<C>(H);
    const ParamLayout L = param_layout(C::T, C::NR, C::NA, C::KR, C::KA, C::H4, H);
    const int nA = C::T * C::T * C::NA * C::KA;
    for (int x = tid; x < nA; x += nthr) {
        int pair = x / (C::NA * C::KA), r = x % (C::NA * C::KA);
        sm[s.cA + pair * C::SA + r] = prm[L.off_cA + x];
        sm[s.cA2 + pair * C::SA + pair_index<C::KA>(r / C::KA, r % C::KA)] = prm[L.off_cA + x];
    }
    if (C::NA % 2)   // the partner of an odd last row is zero
        for (int x = tid; x < C::T * C::T * C::KA; x += nthr)
            sm[s.cA2 + (x / C::KA) * C::SA + pair_index<C::KA>(C::NA, x % C::KA)] = 0.0f;
    const int nR = C::T * C::T * C::NR * C::KR;
    for (int x = tid; x < nR; x += nthr) {
        int pair = x / (C::NR * C::KR), r = x % (C::NR * C::KR);
        sm[s.cR + pair * C::SR + r] = prm[L.off_cR + x];
    }
    const int HD = H * C::D;
    for (int x = tid; x < C::T * H * C::DW; x += nthr) {
        const int t = x / (H * C::DW), r = x % (H * C::DW), h = r / C::DW, d = r % C::DW;
        sm[s.W0 + t * s.SW + r] = d < C::D ? prm[t * L.mlp_stride + h * C::D + d] : 0.0f;
    }
    for (int x = tid; x < C::T * H; x += nthr) {
        int t = x / H, h = x % H;
        sm[s.b0 + t * s.HS + h] = prm[t * L.mlp_stride + HD + h];
        sm[s.w1 + t * s.HS + h] = prm[t * L.mlp_stride + HD + H + h];
    }
    for (int t = tid; t < C::T; t += nthr) sm[s.b1 + t] = prm[t * L.mlp_stride + HD + 2 * H];
}

struct AtomFrame {
    float4 pi;
    int ti;
    float Lx, Ly, Lz, iLx, iLy, iLz;
};

NEP_HD AtomFrame atom_frame(const EvalArgs& a, int i) {
    AtomFrame f;
    f.pi = a.pos4[i];
    f.ti = f2i(f.pi.w);
    const int b = a.cfg[i];
    f.Lx = a.box[3 * b + 0];
    f.Ly = a.box[3 * b + 1];
    f.Lz = a.box[3 * b + 2];
    f.iLx = 1.0f / f.Lx;
    f.iLy = 1.0f / f.Ly;
    f.iLz = 1.0f / f.Lz;
    return f;
}

// Walk over one atom's neighbour entries (slot-major arrays nb / sh, entry
// s of atom i at s * N + i) with the gathers in flight ahead of use:
// neighbour indices DEPTH + 1 entries ahead, their positions (and image
// shifts) DEPTH entries ahead.  Every index read stays below cnt.
template <bool MINIMG, int DEPTH>
struct NbrStream {
    int j[DEPTH + 1];    // entries s .. s + DEPTH
    float4 p[DEPTH];     // entries s .. s + DEPTH - 1
    int sh[DEPTH];
    const int* nb;
    const int* shp;
    NEP_HD NbrStream(const EvalArgs& a, const int* nb_, const int* sh_, int i, int cnt) : nb(nb_), shp(sh_) {
        const int N = a.N;
#pragma unroll
        for (int d = 0; d <= DEPTH; ++d) j[d] = cnt > d ? nb[d * N + i] : 0;
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) {
            p[d] = a.pos4[j[d]];
            sh[d] = (!MINIMG && cnt > d) ? shp[d * N + i] : 0;
        }
    }
    // move from entry s to entry s + 1
    NEP_HD void advance(const EvalArgs& a, int i, int cnt, int s) {
        const int N = a.N;
#pragma unroll
        for (int d = 0; d + 1 < DEPTH; ++d) {
            p[d] = p[d + 1];
            sh[d] = sh[d + 1];
        }
#pragma unroll
        for (int d = 0; d < DEPTH; ++d) j[d] = j[d + 1];
        if (s + DEPTH < cnt) {
            p[DEPTH - 1] = a.pos4[j[DEPTH - 1]];
            if (!MINIMG) sh[DEPTH - 1] = shp[(s + DEPTH) * N + i];
        }
        if (s + DEPTH + 1 < cnt) j[DEPTH] = nb[(s + DEPTH + 1) * N + i];
    }
};

#ifndef NEP_RADIAL_DEPTH
#define NEP_RADIAL_DEPTH 1
#endif
#ifndef NEP_FINISH_DEPTH
#define NEP_FINISH_DEPTH 1
#endif

// ---------------------------------------------------------------------------
// radial descriptor sums and pair compaction, one atom
// ---------------------------------------------------------------------------
// COMPR: the training variant, which also writes the compacted records of
// the pairs inside rc_rad and the mask of the incoming angular slots
template <class C, bool MINIMG, bool COMPR>
NEP_HD void radial_atom(const EvalArgs& a, int i) {
    constexpr int KR = C::KR, T = C::T;
    const int N = a.N;
    const AtomFrame fr = atom_frame(a, i);
    const float rcR2 = a.rc_rad * a.rc_rad, rcA2 = a.rc_ang * a.rc_ang;
    const float irR = 1.0f / a.rc_rad;
    // F[t][k] = sum_{j of species t} Q_k(r_ij)
    float fb[T][KR];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < KR; ++k) fb[t][k] = 0.0f;
    const int cnt = a.cnt[i], cnt_ang = a.cnt_ang[i];
    int nc = 0, ncr = 0, nr = 0;
    unsigned long long amask = 0ull;   // COMPR only
    NbrStream<MINIMG, NEP_RADIAL_DEPTH> ns(a, a.nbr, a.shift, i, cnt);
    for (int s = 0; s < cnt; ++s) {
        const int j = ns.j[0];
        const float4 pj = ns.p[0];
        const int sh = ns.sh[0];
        ns.advance(a, i, cnt, s);
        float dx, dy, dz;
        pair_vector(fr.pi, pj, fr.Lx, fr.Ly, fr.Lz, fr.iLx, fr.iLy, fr.iLz, MINIMG, sh, dx, dy, dz);
        const float d2 = dist2(dx, dy, dz);
        const int tj = f2i(pj.w);
        if (d2 < rcR2) {
            if (COMPR) {
                a.compr[ncr * N + i] = make_float4(dx, dy, dz, i2f((int)(((unsigned)j << 2) | (unsigned)tj)));
                ++ncr;
            }
            if (!COMPR && s >= cnt_ang && a.rin) {
                a.rin[nr * N + i] = j;
                if (!MINIMG) a.rin_sh[nr * N + i] = sh;
                ++nr;
            }
            float f[KR];
            basis<KR>(dist_r(d2), irR, f);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float w = (tj == t) ? 1.0f : 0.0f;
                const float2 w2 = make_float2(w, w);
#pragma unroll
                for (int k = 0; k + 1 < KR; k += 2) {
                    const float2 v = ffma2(w2, make_float2(f[k], f[k + 1]), make_float2(fb[t][k], fb[t][k + 1]));
                    fb[t][k] = v.x;
                    fb[t][k + 1] = v.y;
                }
                if (KR % 2) fb[t][KR - 1] = fmaf(w, f[KR - 1], fb[t][KR - 1]);
            }
        }
        if (s < cnt_ang) {
            const int addr = a.rev[s * N + i] * N + j;
            if (d2 < rcA2) {
                a.comp[nc * N + i] =
                    make_float4(dx, dy, dz, i2f((int)(((unsigned)addr << 2) | (unsigned)tj)));
                ++nc;
                if (COMPR && s < 64) amask |= 1ull << s;
            } else if (COMPR && s >= 64) {
                // the compacted-record force pass reads every angular slot
                // from 64 on and the masked ones below; the list walk of
                // k_finish reads only the slots inside rc_A
                a.fin[addr] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
    }
    a.cnt_comp[i] = nc;
    if (COMPR) {
        a.cnt_compr[i] = ncr;
        a.amask[i] = amask;
    } else if (a.rin) {
        a.cnt_rin[i] = nr;
    }
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < KR; ++k) a.fb[(t * KR + k) * N + i] = fb[t][k];
}

// ---------------------------------------------------------------------------
// angular pieces shared by the fused and the mixed-precision kernels
// ---------------------------------------------------------------------------
// q_n = sum_t sum_k cR[Zi][t][n][k] F[t][k] (Eq. 11 with species-resolved sums)
// row of K floats from shared memory, 16-byte loads when K is a multiple of 4
template <int K>
NEP_HD void load_row(const float* p, float* out) {
    if (K % 4 == 0) {
#pragma unroll
        for (int k = 0; k < K; k += 4) {
            const float4 v = ld4(p + k);
            out[k] = v.x; out[k + 1] = v.y; out[k + 2] = v.z; out[k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = p[k];
    }
}

template <class C>
NEP_HD void radial_q(const EvalArgs& a, const float* sm, const SmemLayout& sl, int ti, int i, float* q) {
    constexpr int NR = C::NR, KR = C::KR, T = C::T;
    const int N = a.N;
    float fbv[T][KR];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < KR; ++k) fbv[t][k] = a.fb[(t * KR + k) * N + i];
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float* c = sm + sl.cR + (ti * T + t) * C::SR + n * KR;
            float cv[KR];
            load_row<KR>(c, cv);
#pragma unroll
            for (int k = 0; k < KR; ++k) acc = fmaf(cv[k], fbv[t][k], acc);
        }
        q[n] = acc;
        NEP_SCHED_BARRIER();
    }
}

// S_nlm = sum_j g_n(r_ij) P_lm(rhat_ij) over the compacted angular pairs
template <class C>
NEP_HD void angular_S(const EvalArgs& a, const float* sm, const SmemLayout& sl, int ti, int i,
                      float (&S)[C::NA][kLM]) {
    constexpr int NA = C::NA, KA = C::KA, T = C::T;
    const int N = a.N;
    const float irA = 1.0f / a.rc_ang;
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int m = 0; m < kLM; ++m) S[n][m] = 0.0f;
    const int nc = a.cnt_comp[i];
    float4 e_nx = nc > 0 ? a.comp[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int c = 0; c < nc; ++c) {
        const float4 e = e_nx;
        if (c + 1 < nc) e_nx = a.comp[(c + 1) * N + i];
        const int tj = f2i(e.w) & 3;
        float r, ir;
        dist_rinv(dist2(e.x, e.y, e.z), r, ir);
        float f[KA];
        basis<KA>(r, irA, f);
        float g[NA];
        contract_pairs<NA, KA>(sm + sl.cA2 + (ti * T + tj) * C::SA, f, g);
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        // S[n][m] += g_n Y_m, two m at a time (paired FMAs)
        float2 gb[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) gb[n] = make_float2(g[n], g[n]);
#pragma unroll
        for (int m = 0; m < kLM; m += 2) {
            float Y0, Y1, gx, gy, gz;
            harm_m(m, ht, Y0, gx, gy, gz);
            harm_m(m + 1, ht, Y1, gx, gy, gz);
            const float2 y2 = make_float2(Y0, Y1);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                const float2 s2 = ffma2(gb[n], y2, make_float2(S[n][m], S[n][m + 1]));
                S[n][m] = s2.x;
                S[n][m + 1] = s2.y;
            }
        }
    }
}

// q_nl = sum_m C_lm S_nlm^2 (Eq. 17) and q4_n = tr(A_n^3)
template <class C>
NEP_HD void angular_q(const float (&S)[C::NA][kLM], float* q) {
    constexpr int NR = C::NR, NA = C::NA;
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float ql[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int m = 0; m < 3; ++m) ql[0] = fmaf(clm(m) * S[n][m], S[n][m], ql[0]);
#pragma unroll
        for (int m = 3; m < 8; ++m) ql[1] = fmaf(clm(m) * S[n][m], S[n][m], ql[1]);
#pragma unroll
        for (int m = 8; m < 15; ++m) ql[2] = fmaf(clm(m) * S[n][m], S[n][m], ql[2]);
#pragma unroll
        for (int m = 15; m < 24; ++m) ql[3] = fmaf(clm(m) * S[n][m], S[n][m], ql[3]);
#pragma unroll
        for (int l = 0; l < 4; ++l) q[NR + n * 4 + l] = ql[l];
        if (C::H4) {
            const float s2[5] = {S[n][3], S[n][4], S[n][5], S[n][6], S[n][7]};
            q[NR + NA * 4 + n] = fourbody<float>(s2, nullptr);
        }
    }
}

// dE_i/dS_nlm = 2 C_lm S_nlm dE/dq_nl (+ the 4-body chain through l = 2);
// S(n, m) and pl(n, l) are the atom's S and angular dE/dq
template <class C, class GetS, class GetP>
NEP_HD void make_Sb(float (&Sb)[C::NA][kLM], GetS S, GetP pl) {
    constexpr int NA = C::NA;
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float s2[5];
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            const float s = S(n, m);
            if (m >= 3 && m < 8) s2[m - 3] = s;
            Sb[n][m] = 2.0f * clm(m) * pl(n, lm_l(m) - 1) * s;
        }
        if (C::H4) {
            const float p4 = pl(n, 4);
            float ds[5];
            fourbody(s2, ds);
#pragma unroll
            for (int m = 0; m < 5; ++m) Sb[n][3 + m] = fmaf(p4, ds[m], Sb[n][3 + m]);
        }
    }
}

// angular pair forces: f_ij = u sum_m (b_m - l a_m / r) Y_m + (1/r) sum_m a_m grad P_m(u),
// a_m = sum_n Sb[n][m] g_n, b_m = sum_n Sb[n][m] g'_n; owner sums and reverse-slot scatter
// SPLIT: sum (b_m - l a_m / r) Y_m and a_m grad P_m as even and odd partial
// sums over m, one paired FMA per pair of m (measured faster in the
// tensor-core kernel, slower in the FP32 one)
template <class C, bool SPLIT = false>
NEP_HD void angular_force(const EvalArgs& a, const float* sm, const SmemLayout& sl, int ti, int i,
                          const float (&Sb)[C::NA][kLM], float& Fx, float& Fy, float& Fz, float* W) {
    constexpr int NA = C::NA, KA = C::KA, T = C::T;
    const int N = a.N;
    const float irA = 1.0f / a.rc_ang;
    const int nc = a.cnt_comp[i];
    float4 e_nx = nc > 0 ? a.comp[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int c = 0; c < nc; ++c) {
        const float4 e = e_nx;
        if (c + 1 < nc) e_nx = a.comp[(c + 1) * N + i];
        const int bits = f2i(e.w);
        const int tj = bits & 3;
        const int addr = (int)((unsigned)bits >> 2);
        float r, ir;
        dist_rinv(dist2(e.x, e.y, e.z), r, ir);
        float g[NA], gp[NA];
        {
            float f[KA], fp[KA];
            basis_d<KA>(r, irA, f, fp);
            const float* c2 = sm + sl.cA2 + (ti * T + tj) * C::SA;
            contract_pairs<NA, KA>(c2, f, g);
            contract_pairs<NA, KA>(c2, fp, gp);
        }
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        float rad = 0.0f, Gx = 0.0f, Gy = 0.0f, Gz = 0.0f;
        float2 rad2 = make_float2(0.0f, 0.0f), gx2 = rad2, gy2 = rad2, gz2 = rad2;
        // a_m and b_m two m at a time (paired FMAs, each chain in n order)
        float2 gb[NA], gpb[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            gb[n] = make_float2(g[n], g[n]);
            gpb[n] = make_float2(gp[n], gp[n]);
        }
#pragma unroll
        for (int m0 = 0; m0 < kLM; m0 += 2) {
            float2 am2 = make_float2(0.0f, 0.0f), bm2 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                const float2 s2 = make_float2(Sb[n][m0], Sb[n][m0 + 1]);
                am2 = ffma2(s2, gb[n], am2);
                bm2 = ffma2(s2, gpb[n], bm2);
            }
            if constexpr (SPLIT) {
                float Y0, hx0, hy0, hz0, Y1, hx1, hy1, hz1;
                harm_m(m0, ht, Y0, hx0, hy0, hz0);
                harm_m(m0 + 1, ht, Y1, hx1, hy1, hz1);
                const float2 cl = make_float2(-(float)lm_l(m0) * ir, -(float)lm_l(m0 + 1) * ir);
                rad2 = ffma2(ffma2(cl, am2, bm2), make_float2(Y0, Y1), rad2);
                gx2 = ffma2(am2, make_float2(hx0, hx1), gx2);
                gy2 = ffma2(am2, make_float2(hy0, hy1), gy2);
                gz2 = ffma2(am2, make_float2(hz0, hz1), gz2);
            } else {
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int m = m0 + u;
                    const float am = u ? am2.y : am2.x, bm = u ? bm2.y : bm2.x;
                    float Y, hx, hy, hz;
                    harm_m(m, ht, Y, hx, hy, hz);
                    rad = fmaf(fmaf(-(float)lm_l(m) * ir, am, bm), Y, rad);
                    Gx = fmaf(am, hx, Gx);
                    Gy = fmaf(am, hy, Gy);
                    Gz = fmaf(am, hz, Gz);
                }
            }
        }
        if constexpr (SPLIT) {
            rad = rad2.x + rad2.y;
            Gx = gx2.x + gx2.y;
            Gy = gy2.x + gy2.y;
            Gz = gz2.x + gz2.y;
        }
        const float fx = fmaf(ht.x, rad, Gx * ir);
        const float fy = fmaf(ht.y, rad, Gy * ir);
        const float fz = fmaf(ht.z, rad, Gz * ir);
        Fx += fx; Fy += fy; Fz += fz;
        W[0] -= fx * e.x; W[1] -= fx * e.y; W[2] -= fx * e.z;
        W[3] -= fy * e.x; W[4] -= fy * e.y; W[5] -= fy * e.z;
        W[6] -= fz * e.x; W[7] -= fz * e.y; W[8] -= fz * e.z;
        a.fin[addr] = make_float4(fx, fy, fz, 0.0f);
    }
}

// per-species network: E = sum_h w1 tanh(W0 q + b0) + b1, p = dE/dq;
// writes E, the species-projected radial adjoint P[i][t][k] = sum_n p_n cR[Zi][t][n][k]
template <class C>
NEP_HD void network(const EvalArgs& a, const float* sm, const SmemLayout& sl, int ti, int i,
                    const float* q, float* p) {
    constexpr int NR = C::NR, KR = C::KR, T = C::T, D = C::D, DW = C::DW;
    const float* W0 = sm + sl.W0 + ti * sl.SW;
    const float* b0 = sm + sl.b0 + ti * sl.HS;
    const float* w1 = sm + sl.w1 + ti * sl.HS;
    float E = sm[sl.b1 + ti];
    float qv[DW], pv[DW];
#pragma unroll
    for (int d = 0; d < DW; ++d) {
        qv[d] = d < D ? q[d] : 0.0f;
        pv[d] = 0.0f;
    }
    for (int h = 0; h < a.H; ++h) {
        float w[DW];
        load_row<DW>(W0 + h * DW, w);
        // W0 q as two interleaved partial sums (even and odd d) in paired FMAs
        float2 z2 = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int d = 0; d < DW; d += 2)
            z2 = ffma2(make_float2(w[d], w[d + 1]), make_float2(qv[d], qv[d + 1]), z2);
        const float z = b0[h] + (z2.x + z2.y);
        const float t = tanh_f(z);
        const float wh = w1[h];
        E = fmaf(wh, t, E);
        const float sg = wh * (1.0f - t * t);
        const float2 sg2 = make_float2(sg, sg);
        static_assert(DW % 2 == 0, "W0 rows are padded to a multiple of 4");
#pragma unroll
        for (int d = 0; d < DW; d += 2) {
            const float2 v = ffma2(sg2, make_float2(w[d], w[d + 1]), make_float2(pv[d], pv[d + 1]));
            pv[d] = v.x;
            pv[d + 1] = v.y;
        }
    }
#pragma unroll
    for (int d = 0; d < D; ++d) p[d] = pv[d];
    a.e_atom[i] = E;
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float* c = sm + sl.cR + (ti * T + t) * C::SR;
        float acc[KR];
#pragma unroll
        for (int k = 0; k < KR; ++k) acc[k] = 0.0f;
#pragma unroll
        for (int n = 0; n < NR; ++n) {
            float cv[KR];
            load_row<KR>(c + n * KR, cv);
#pragma unroll
            for (int k = 0; k < KR; ++k) acc[k] = fmaf(p[n], cv[k], acc[k]);
        }
        if (KR % 4 == 0) {
            float4* dst = reinterpret_cast<float4*>(a.Pr + (i * T + t) * KR);
#pragma unroll
            for (int k = 0; k < KR; k += 4) dst[k / 4] = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < KR; ++k) a.Pr[(i * T + t) * KR + k] = acc[k];
        }
        NEP_SCHED_BARRIER();
    }
}

// ---------------------------------------------------------------------------
// fused angular descriptor + network + angular forces, one atom.  `stage`
// points at this thread's column of a [NA*24][blockDim] shared array where S
// waits while the network runs (stride `sstride` floats between entries).
// ---------------------------------------------------------------------------
template <class C>
NEP_HD void angular_atom(const EvalArgs& a, const float* sm, float* stage, int sstride, int i) {
    constexpr int NR = C::NR, NA = C::NA, D = C::D;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N;
    const int ti = f2i(a.pos4[i].w);
    float q[D];
    radial_q<C>(a, sm, sl, ti, i, q);
    {
        float S[NA][kLM];
        angular_S<C>(a, sm, sl, ti, i, S);
        angular_q<C>(S, q);
        if (a.S) {
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int m = 0; m < kLM; ++m) a.S[(n * kLM + m) * N + i] = S[n][m];
        }
#pragma unroll
        for (int n = 0; n < NA; ++n)
#pragma unroll
            for (int m = 0; m < kLM; ++m) stage[(n * kLM + m) * sstride] = S[n][m];
    }
    float p[D];
    network<C>(a, sm, sl, ti, i, q, p);
    if (a.q_out) {
#pragma unroll
        for (int d = 0; d < D; ++d) a.q_out[d * N + i] = q[d];
    }
    if (a.p_out) {
#pragma unroll
        for (int d = 0; d < D; ++d) a.p_out[d * N + i] = p[d];
    }
    float Sb[NA][kLM];
    make_Sb<C>(Sb, [&](int n, int m) { return stage[(n * kLM + m) * sstride]; },
               [&](int n, int l) { return p[NR + (l < 4 ? n * 4 + l : NA * 4 + n)]; });
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    float W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = 0.0f;
    angular_force<C>(a, sm, sl, ti, i, Sb, Fx, Fy, Fz, W);
    a.fpart[i] = Fx;
    a.fpart[N + i] = Fy;
    a.fpart[2 * N + i] = Fz;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.wat[k * N + i] = W[k];
}

// The same atom with S_nlm parked in the thread's TMEM lane (tS: column 0 of
// the lane) while the network runs.  Every thread of the warp calls it (the
// TMEM moves are warp-collective); `valid` guards the atom's own work.
template <class C>
__device__ void angular_atom_tm(const EvalArgs& a, const float* sm, uint32_t tS, int i, bool valid) {
    constexpr int NR = C::NR, NA = C::NA, D = C::D;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N;
    const int ti = valid ? f2i(a.pos4[i].w) : 0;
    float q[D];
    {
        float S[NA][kLM];
        if (valid) {
            radial_q<C>(a, sm, sl, ti, i, q);
            angular_S<C>(a, sm, sl, ti, i, S);
        } else {
#pragma unroll
            for (int d = 0; d < D; ++d) q[d] = 0.0f;
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int m = 0; m < kLM; ++m) S[n][m] = 0.0f;
        }
        angular_q<C>(S, q);
        if (valid && a.S) {
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int m = 0; m < kLM; ++m) a.S[(n * kLM + m) * N + i] = S[n][m];
        }
        __syncwarp();
        const float* Sf = &S[0][0];
#pragma unroll
        for (int c = 0; c < NA * kLM; c += 8) tc5::st8(tS + c, Sf + c);
    }
    float p[D];
    if (valid) {
        network<C>(a, sm, sl, ti, i, q, p);
        if (a.q_out) {
#pragma unroll
            for (int d = 0; d < D; ++d) a.q_out[d * N + i] = q[d];
        }
        if (a.p_out) {
#pragma unroll
            for (int d = 0; d < D; ++d) a.p_out[d * N + i] = p[d];
        }
    } else {
#pragma unroll
        for (int d = 0; d < D; ++d) p[d] = 0.0f;
    }
    float Sb[NA][kLM];
    __syncwarp();
    tc5::wait_st();
    {
        float* Sf = &Sb[0][0];
#pragma unroll
        for (int c = 0; c < NA * kLM; c += 8) tc5::ld8(tS + c, Sf + c);
        tc5::wait_ld();
    }
    if (!valid) return;
    make_Sb<C>(Sb, [&](int n, int m) { return Sb[n][m]; },
               [&](int n, int l) { return p[NR + (l < 4 ? n * 4 + l : NA * 4 + n)]; });
    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    float W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = 0.0f;
    angular_force<C>(a, sm, sl, ti, i, Sb, Fx, Fy, Fz, W);
    a.fpart[i] = Fx;
    a.fpart[N + i] = Fy;
    a.fpart[2 * N + i] = Fz;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.wat[k * N + i] = W[k];
}

// ---------------------------------------------------------------------------
// radial pair forces of both directions: dE_i/dr_ij + dE_j/dr_ij along rhat,
// from P of atom i (neighbour species row) and P of atom j (row Zi); returns
// F_i's radial part and the symmetric radial virial (xx yy zz xy xz yz)
// ---------------------------------------------------------------------------
// stage (optional): this thread's slot of a [T*KR/4][nthr] float4 array in
// shared memory; the atom's own adjoint rows are kept there instead of in
// T*KR registers and read per pair for the neighbour's species
// COMPR: the training variant, which walks the compacted records of the
// radial kernel instead of the list
template <class C, bool MINIMG, bool COMPR>
NEP_HD void radial_force_atom(const EvalArgs& a, int i, float& Fx, float& Fy, float& Fz, float* Wr,
                              float4* stage = nullptr, int nthr = 0) {
    constexpr int KR = C::KR, T = C::T;
    const int N = a.N;
    const AtomFrame fr = atom_frame(a, i);
    const int ti = fr.ti;
    const float rcR2 = a.rc_rad * a.rc_rad;
    const float irR = 1.0f / a.rc_rad;
    constexpr bool kStageable = (KR % 4) == 0;
    const bool staged = kStageable && stage != nullptr;
    float Pi[T][KR];
    if (staged) {
        const float4* src = reinterpret_cast<const float4*>(a.Pr + i * T * KR);
#pragma unroll
        for (int c = 0; c < T * KR / 4; ++c) stage[c * nthr] = src[c];
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int k = 0; k < KR; ++k) Pi[t][k] = 0.0f;
    } else if ((T * KR) % 4 == 0) {
        const float4* src = reinterpret_cast<const float4*>(a.Pr + i * T * KR);
#pragma unroll
        for (int x = 0; x < T * KR; x += 4) {
            const float4 v = src[x / 4];
            Pi[x / KR][x % KR] = v.x;
            Pi[(x + 1) / KR][(x + 1) % KR] = v.y;
            Pi[(x + 2) / KR][(x + 2) % KR] = v.z;
            Pi[(x + 3) / KR][(x + 3) % KR] = v.w;
        }
    } else {
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int k = 0; k < KR; ++k) Pi[t][k] = a.Pr[(i * T + t) * KR + k];
    }
    // one pair: both directions of the radial force along r_ij, and the
    // owner's symmetric radial virial
    auto pair = [&](int j, int tj, float dx, float dy, float dz, float d2) {
        float r, ir;
        dist_rinv(d2, r, ir);
        float f[KR], fp[KR];
        basis_d<KR>(r, irR, f, fp);
        float Pj[KR];
        if (KR % 8 == 0) {
            // rows of K_R floats start on 32-byte boundaries (256-byte aligned base)
#pragma unroll
            for (int k = 0; k < KR; k += 8) load8_ro(a.Pr + (j * T + ti) * KR + k, Pj + k);
        } else if (KR % 4 == 0) {
            const float4* src = reinterpret_cast<const float4*>(a.Pr + (j * T + ti) * KR);
#pragma unroll
            for (int k = 0; k < KR; k += 4) {
                const float4 v = src[k / 4];
                Pj[k] = v.x; Pj[k + 1] = v.y; Pj[k + 2] = v.z; Pj[k + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < KR; ++k) Pj[k] = a.Pr[(j * T + ti) * KR + k];
        }
        float dEi = 0.0f, dEj = 0.0f;
        if (kStageable && staged) {
#pragma unroll
            for (int c = 0; c < KR / 4; ++c) {
                const float4 v = stage[(tj * (KR / 4) + c) * nthr];
                const float pv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    dEi = fmaf(pv[u], fp[4 * c + u], dEi);
                    dEj = fmaf(Pj[4 * c + u], fp[4 * c + u], dEj);
                }
            }
        } else {
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                float pk = Pi[0][k];
#pragma unroll
                for (int t = 1; t < T; ++t) pk = (tj == t) ? Pi[t][k] : pk;
                dEi = fmaf(pk, fp[k], dEi);
                dEj = fmaf(Pj[k], fp[k], dEj);
            }
        }
        const float tot = (dEi + dEj) * ir;
        Fx = fmaf(tot, dx, Fx); Fy = fmaf(tot, dy, Fy); Fz = fmaf(tot, dz, Fz);
        const float w = dEi * ir;
        const float wx = w * dx, wy = w * dy, wz = w * dz;
        Wr[0] = fmaf(wx, dx, Wr[0]); Wr[1] = fmaf(wy, dy, Wr[1]); Wr[2] = fmaf(wz, dz, Wr[2]);
        Wr[3] = fmaf(wx, dy, Wr[3]); Wr[4] = fmaf(wx, dz, Wr[4]); Wr[5] = fmaf(wy, dz, Wr[5]);
    };
    if (COMPR) {
        // pairs inside rc_rad, compacted by the radial kernel
        const int ncr = a.cnt_compr[i];
        float4 q_nx = ncr > 0 ? a.compr[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
        for (int s = 0; s < ncr; ++s) {
            const float4 e = q_nx;
            if (s + 1 < ncr) q_nx = a.compr[(s + 1) * N + i];
            const int bits = f2i(e.w);
            pair((int)((unsigned)bits >> 2), bits & 3, e.x, e.y, e.z, dist2(e.x, e.y, e.z));
        }
        // incoming angular pair forces: the prefix slots inside rc_A (the
        // mask, in batches of four independent loads, ascending) and every
        // slot from 64 on; without a mask every slot of the prefix
        const int na = a.cnt_ang[i];
        const int s0 = na < 64 ? na : 64;
        {
            unsigned long long m = a.amask[i];
            while (m) {
                int sl[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    sl[u] = m ? low_bit(m) : -1;
                    m &= m - 1ull;
                }
                float4 g[4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    g[u] = sl[u] >= 0 ? a.fin[(size_t)sl[u] * N + i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (sl[u] >= 0) { Fx -= g[u].x; Fy -= g[u].y; Fz -= g[u].z; }
                }
            }
        }
        for (int s = s0; s < na; ++s) {
            const float4 g = a.fin[(size_t)s * N + i];
            Fx -= g.x; Fy -= g.y; Fz -= g.z;
        }
        return;
    }
    // Walk 1, the angular prefix: radial pairs, and which prefix slots lie
    // inside rc_A.  The pair vector seen from j is the exact negation of the
    // one seen from i, so j's angular kernel wrote the incoming force of slot
    // s exactly when d2 < rc_A^2 here; only those slots are read.  Slots
    // below 64 are marked in a bit mask and read afterwards in batches of
    // four independent loads, ascending; any later slot is read in the walk.
    // Walk 2: the entries after the prefix that the radial kernel found
    // inside rc_rad (the shell beyond rc_rad is not visited again), or with
    // no skin simply the rest of the list.
    const float rcA2 = a.rc_ang * a.rc_ang;
    const int cnt_ang = a.cnt_ang[i];
    unsigned long long amask = 0ull;
    {
        NbrStream<MINIMG, NEP_FINISH_DEPTH> ns(a, a.nbr, a.shift, i, cnt_ang);
        for (int s = 0; s < cnt_ang; ++s) {
            const int j = ns.j[0];
            const float4 pj = ns.p[0];
            const int sh = ns.sh[0];
            ns.advance(a, i, cnt_ang, s);
            float dx, dy, dz;
            pair_vector(fr.pi, pj, fr.Lx, fr.Ly, fr.Lz, fr.iLx, fr.iLy, fr.iLz, MINIMG, sh, dx, dy, dz);
            const float d2 = dist2(dx, dy, dz);
            if (d2 < rcA2) {
                if (s < 64) {
                    amask |= 1ull << s;
                } else {
                    const float4 g = a.fin[(size_t)s * N + i];
                    Fx -= g.x; Fy -= g.y; Fz -= g.z;
                }
            }
            if (d2 < rcR2) pair(j, f2i(pj.w), dx, dy, dz, d2);
        }
    }
    {
        // without a skin the rest of the list is the set inside rc_rad itself
        const int* nb2 = a.rin ? a.rin : a.nbr + (size_t)cnt_ang * N;
        const int* sh2 = a.rin ? a.rin_sh : (a.shift ? a.shift + (size_t)cnt_ang * N : nullptr);
        const int nr = a.rin ? a.cnt_rin[i] : a.cnt[i] - cnt_ang;
        NbrStream<MINIMG, NEP_FINISH_DEPTH> ns(a, nb2, sh2, i, nr);
        for (int s = 0; s < nr; ++s) {
            const int j = ns.j[0];
            const float4 pj = ns.p[0];
            const int sh = ns.sh[0];
            ns.advance(a, i, nr, s);
            float dx, dy, dz;
            pair_vector(fr.pi, pj, fr.Lx, fr.Ly, fr.Lz, fr.iLx, fr.iLy, fr.iLz, MINIMG, sh, dx, dy, dz);
            const float d2 = dist2(dx, dy, dz);
            if (d2 < rcR2) pair(j, f2i(pj.w), dx, dy, dz, d2);
        }
    }
    while (amask) {
        int sl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            sl[u] = amask ? low_bit(amask) : -1;
            amask &= amask - 1ull;
        }
        float4 g[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            g[u] = sl[u] >= 0 ? a.fin[(size_t)sl[u] * N + i] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (sl[u] >= 0) { Fx -= g[u].x; Fy -= g[u].y; Fz -= g[u].z; }
        }
    }
}

// F_i = radial part + angular owner part - sum of the scattered incoming
// angular pair forces (subtracted inside radial_force_atom); the per-atom
// virial (angular owner part minus the radial part) is written back for the
// per-configuration reduction
template <class C, bool MINIMG, bool COMPR>
NEP_HD void finish_atom(const EvalArgs& a, int i, float* force, float* e_out, float4* stage = nullptr,
                        int nthr = 0) {
    const int N = a.N;
    float Fx = a.fpart[i], Fy = a.fpart[N + i], Fz = a.fpart[2 * N + i];
    float Wr[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    radial_force_atom<C, MINIMG, COMPR>(a, i, Fx, Fy, Fz, Wr, stage, nthr);
    force[i] = Fx;
    force[N + i] = Fy;
    force[2 * N + i] = Fz;
    if (e_out) e_out[i] = a.e_atom[i];
    const float Wsym[9] = {Wr[0], Wr[3], Wr[4], Wr[3], Wr[1], Wr[5], Wr[4], Wr[5], Wr[2]};
#pragma unroll
    for (int c = 0; c < 9; ++c) a.wat[(size_t)c * N + i] -= Wsym[c];
}

// ---------------------------------------------------------------------------
// kernels and launchers
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
// Resident blocks per SM that the register allocation of k_angular is sized
// for (65536 / (128 x MINB) registers per thread: 255, 168 or 128).  It is
// compiled for MINB = 2, 3 and 4; the runtime picks one per system size class
// (nep_autotune).  Variant 0 (255 registers) keeps S and dE/dS on chip
// without spills and is the default.
NEP_HD constexpr int variant_minb(int v) { return v + 2; }
// Default block sizes of the radial and finish kernels; the autotuner may
// pick another of kBlockChoices per size class.  Each size keeps the
// kernel at 64 registers (1,024 / block resident blocks).
constexpr int kRadialBlock = 256;
constexpr int kFinishThreads = 128;

#ifndef NEP_RADIAL_MINB
#define NEP_RADIAL_MINB 4
#endif
#ifndef NEP_FINISH_MINB
#define NEP_FINISH_MINB 8
#endif
#ifndef NEP_FINISH_STAGE
#define NEP_FINISH_STAGE 1
#endif
template <class C, bool MINIMG, bool COMPR, int BLOCK = kRadialBlock>
__global__ void __launch_bounds__(BLOCK, NEP_RADIAL_MINB * kRadialBlock / BLOCK) k_radial(const EvalArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N) radial_atom<C, MINIMG, COMPR>(a, i);
}

// Persistent: one CTA per resident slot, the model image staged once, then a
// grid-stride loop over tiles of 128 atoms.
// The 255-register variant (MINB 2) parks S_nlm in tensor memory, NA x 24
// columns per CTA; the others stage it in shared memory.
template <int MINB>
NEP_HD constexpr bool angular_uses_tmem() { return MINB == 2; }
template <class C>
NEP_HD constexpr uint32_t angular_tmem_cols() { return tc5::tmem_cols(C::NA * kLM); }

template <class C, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_angular(const EvalArgs a) {
    extern __shared__ float sm[];
    const SmemLayout sl = smem_layout<C>(a.H);
    load_model<C>(sm, a.params, a.H, threadIdx.x, blockDim.x);
    const int ntiles = (a.N + kBlock - 1) / kBlock;
    if constexpr (angular_uses_tmem<MINB>()) {
        __shared__ uint32_t tslot;
        const int warp = threadIdx.x >> 5;
        if (warp == 0) tc5::alloc(&tslot, angular_tmem_cols<C>());
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        const uint32_t tbase = tslot;
        const uint32_t tS = tc5::lane_addr(tbase, warp, 0);
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int i = tile * kBlock + threadIdx.x;
            angular_atom_tm<C>(a, sm, tS, i, i < a.N);
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        if (warp == 0) tc5::dealloc(tbase, angular_tmem_cols<C>());
    } else {
        __syncthreads();
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const int i = tile * kBlock + threadIdx.x;
            if (i < a.N) angular_atom<C>(a, sm, sm + sl.total + threadIdx.x, kBlock, i);
        }
    }
}

// resident CTAs per SM of a kernel variant, measured once at model creation
template <class C, int MINB, int KIND>
int& resident_blocks() {
    static int b = 1;
    return b;
}
inline int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}
// Resident CTAs per SM of a kernel from its registers (allocated per warp
// in units of 256), shared memory and threads.  The runtime's occupancy
// query reports one CTA per SM for every kernel that allocates tensor
// memory, whatever its resources, so those kernels count here and cap the
// result by their share of the SM's 512 TMEM columns.
inline int resident_by_resources(const void* fn, int threads, size_t dyn_smem, int tmem_cols_per_cta) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 1;
    int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, blk_sm = 0, smem_rsv = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int warps = (threads + 31) / 32;
    const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
    int n = blk_sm;
    if (regs_warp > 0) n = std::min(n, regs_sm / regs_warp / warps);
    const size_t smem_blk = fa.sharedSizeBytes + dyn_smem + (size_t)smem_rsv;
    if (smem_blk > 0) n = std::min(n, (int)((size_t)smem_sm / smem_blk));
    n = std::min(n, thr_sm / threads);
    if (tmem_cols_per_cta > 0) n = std::min(n, 512 / tmem_cols_per_cta);
    return n < 1 ? 1 : n;
}

inline int persistent_grid(int ntiles, int per_sm) {
    const int g = sm_count() * (per_sm > 0 ? per_sm : 1);
    return ntiles < g ? ntiles : g;
}

template <class C, bool MINIMG, int BLOCK = kFinishThreads, bool COMPR = false>
__global__ void __launch_bounds__(BLOCK, NEP_FINISH_MINB * kFinishThreads / BLOCK) k_finish(const EvalArgs a, float* force, float* e_out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
#if NEP_FINISH_STAGE
    constexpr int kChunks = (C::KR % 4 == 0) ? C::T * C::KR / 4 : 1;
    __shared__ float4 stage[kChunks * BLOCK];
    if (i < a.N) finish_atom<C, MINIMG, COMPR>(a, i, force, e_out, stage + threadIdx.x, BLOCK);
#else
    if (i < a.N) finish_atom<C, MINIMG, COMPR>(a, i, force, e_out);
#endif
}

template <class C>
size_t smem_bytes_of(int H) { return sizeof(float) * (size_t)smem_layout<C>(H).total; }
template <class C>
size_t angular_smem_bytes(int H, bool tmem_stage) {
    return sizeof(float) * ((size_t)smem_layout<C>(H).total + (tmem_stage ? 0 : (size_t)C::NA * kLM * kBlock));
}

template <class C, int BLOCK>
void launch_radial_b(const EvalArgs& a, cudaStream_t st) {
    const int grid = (a.N + BLOCK - 1) / BLOCK;
    if (a.min_image)
        k_radial<C, true, false, BLOCK><<<grid, BLOCK, 0, st>>>(a);
    else
        k_radial<C, false, false, BLOCK><<<grid, BLOCK, 0, st>>>(a);
}

// block: one of kBlockChoices, 0 for the default; the training variant
// (compacted records) always runs at the default block
template <class C>
cudaError_t launch_radial_t(const EvalArgs& a, cudaStream_t st, int block) {
    if (a.N == 0) return cudaSuccess;
    if (a.compr) {
        const int grid = (a.N + kRadialBlock - 1) / kRadialBlock;
        if (a.min_image)
            k_radial<C, true, true><<<grid, kRadialBlock, 0, st>>>(a);
        else
            k_radial<C, false, true><<<grid, kRadialBlock, 0, st>>>(a);
    } else if (block == 64) {
        launch_radial_b<C, 64>(a, st);
    } else if (block == 128) {
        launch_radial_b<C, 128>(a, st);
    } else {
        launch_radial_b<C, kRadialBlock>(a, st);
    }
    return cudaGetLastError();
}

template <class C, int MINB>
void launch_angular_v(const EvalArgs& a, cudaStream_t st, int ntiles) {
    const size_t smem = angular_smem_bytes<C>(a.H, angular_uses_tmem<MINB>());
    k_angular<C, MINB><<<persistent_grid(ntiles, resident_blocks<C, MINB, 0>()), kBlock, smem, st>>>(a);
}

template <class C>
cudaError_t launch_angular_t(const EvalArgs& a, cudaStream_t st, int v) {
    const int ntiles = (a.N + kBlock - 1) / kBlock;
    if (ntiles == 0) return cudaSuccess;
    if (v == 1)
        launch_angular_v<C, 3>(a, st, ntiles);
    else if (v == 2)
        launch_angular_v<C, 4>(a, st, ntiles);
    else
        launch_angular_v<C, 2>(a, st, ntiles);
    return cudaGetLastError();
}

template <class C, int BLOCK>
void launch_finish_b(const EvalArgs& a, const FinishArgs& f, cudaStream_t st) {
    const int grid = (a.N + BLOCK - 1) / BLOCK;
    if (a.min_image)
        k_finish<C, true, BLOCK><<<grid, BLOCK, 0, st>>>(a, f.force, f.e_out);
    else
        k_finish<C, false, BLOCK><<<grid, BLOCK, 0, st>>>(a, f.force, f.e_out);
}

// block: one of kBlockChoices, 0 for the default; the training variant
// (compacted records) always runs at the default block
template <class C>
cudaError_t launch_finish_t(const EvalArgs& a, const FinishArgs& f, int max_chunks, cudaStream_t st, int block) {
    if (a.N > 0) {
        if (a.compr) {
            const int grid = (a.N + kFinishThreads - 1) / kFinishThreads;
            if (a.min_image)
                k_finish<C, true, kFinishThreads, true><<<grid, kFinishThreads, 0, st>>>(a, f.force, f.e_out);
            else
                k_finish<C, false, kFinishThreads, true><<<grid, kFinishThreads, 0, st>>>(a, f.force, f.e_out);
        } else if (block == 64)
            launch_finish_b<C, 64>(a, f, st);
        else if (block == 256)
            launch_finish_b<C, 256>(a, f, st);
        else
            launch_finish_b<C, kFinishThreads>(a, f, st);
    }
    return launch_chunk_reduce(a, f, max_chunks, st);
}

// resident CTAs per SM of one angular variant; a variant that parks S in
// tensor memory also fits its allocation into the SM's 512 columns, so that
// no CTA of the persistent grid waits for another one's columns
template <class C, int MINB>
cudaError_t init_v(int H) {
    const int smem = (int)angular_smem_bytes<C>(H, angular_uses_tmem<MINB>());
    cudaError_t e = cudaFuncSetAttribute(k_angular<C, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    sm_count();
    int& rb = resident_blocks<C, MINB, 0>();
    if (angular_uses_tmem<MINB>()) {
        rb = resident_by_resources((const void*)k_angular<C, MINB>, kBlock, smem, (int)angular_tmem_cols<C>());
        return cudaGetLastError();
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rb, k_angular<C, MINB>, kBlock, smem);
}

template <class C>
cudaError_t init_t(int H) {
    cudaError_t e;
    if ((e = init_v<C, 2>(H))) return e;
    if ((e = init_v<C, 3>(H))) return e;
    return init_v<C, 4>(H);
}

#define NEP_DEFINE_KERNEL_SET(NAME, NR, NA, KR, KA, H4, T)                                    \
    extern const KernelSet NAME = {NR, NA, KR, KA, H4, T,                                        \
                                   &smem_bytes_of<Cfg<NR, NA, KR, KA, H4, T>>,                   \
                                   &init_t<Cfg<NR, NA, KR, KA, H4, T>>,                          \
                                   &launch_radial_t<Cfg<NR, NA, KR, KA, H4, T>>,                 \
                                   &launch_angular_any_t<Cfg<NR, NA, KR, KA, H4, T>>,            \
                                   &launch_finish_t<Cfg<NR, NA, KR, KA, H4, T>>,                 \
                                   &train_init_t<Cfg<NR, NA, KR, KA, H4, T>>,                    \
                                   &train_t<Cfg<NR, NA, KR, KA, H4, T>>,                         \
                                   &grad_chunks_t<Cfg<NR, NA, KR, KA, H4, T>>};
#endif

}  // namespace nep
