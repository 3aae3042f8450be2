// Per-atom NEP kernels, templated on the compiled hyper-parameters.
//
//   desc   (one thread per atom i):  radial descriptor via species-resolved
//          basis sums, angular S_nlm (Eq. 16) over the compacted angular
//          pairs, q_nl (Eq. 17), 4-body q4_n, the per-species tanh network
//          (Section 2.3) and dE/dq.
//   force  (one thread per atom i):  f_ij = dE_i/dr_ij for every pair
//          (Eq. 3), radial part for both directions of the pair, angular part
//          scattered to the reverse slot, per-atom virial (Eq. 4).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "nep_device.cuh"

namespace nep {

// Keeps the compiler from hoisting every shared-memory load of a fully
// unrolled contraction ahead of its FMAs (which costs registers and spills).
#if defined(__CUDA_ARCH__)
#define NEP_SCHED_BARRIER() asm volatile("" ::: "memory")
#else
#define NEP_SCHED_BARRIER() ((void)0)
#endif

NEP_HD constexpr int odd_up(int x) { return (x % 2) ? x : x + 1; }
NEP_HD int stride_1mod32(int x) { return x + ((33 - (x % 32)) % 32); }

template <int NR_, int NA_, int KR_, int KA_, int H4_, int T_>
struct Cfg {
    static constexpr int NR = NR_, NA = NA_, KR = KR_, KA = KA_, H4 = H4_, T = T_;
    static constexpr int D = NR + NA * 4 + (H4 ? NA : 0);
    static constexpr int NP = NA * (4 + (H4 ? 1 : 0));   // angular + 4-body descriptor count
    static constexpr int SA = odd_up(NA * KA);           // per-species-pair stride, odd
    static constexpr int SR = odd_up(NR * KR);
};

// Shared-memory image of the model, padded so that the (up to 9) species
// pairs or 3 species met by one warp fall in distinct banks.
struct SmemLayout {
    int cA, cR, W0, b0, w1, b1, total;
    int SW, HS;
};

template <class C>
NEP_HD SmemLayout smem_layout(int H) {
    SmemLayout s;
    s.SW = stride_1mod32(H * C::D);
    s.HS = (H % 2) ? H : H + 1;
    s.cA = 0;
    s.cR = s.cA + C::T * C::T * C::SA;
    s.W0 = s.cR + C::T * C::T * C::SR;
    s.b0 = s.W0 + C::T * s.SW;
    s.w1 = s.b0 + C::T * s.HS;
    s.b1 = s.w1 + C::T * s.HS;
    s.total = s.b1 + C::T;
    return s;
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
    }
    const int nR = C::T * C::T * C::NR * C::KR;
    for (int x = tid; x < nR; x += nthr) {
        int pair = x / (C::NR * C::KR), r = x % (C::NR * C::KR);
        sm[s.cR + pair * C::SR + r] = prm[L.off_cR + x];
    }
    const int HD = H * C::D;
    for (int x = tid; x < C::T * HD; x += nthr) {
        int t = x / HD, r = x % HD;
        sm[s.W0 + t * s.SW + r] = prm[t * L.mlp_stride + r];
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

// ---------------------------------------------------------------------------
// descriptor + network, one atom
// ---------------------------------------------------------------------------
template <class C, bool MINIMG>
NEP_HD void desc_atom(const EvalArgs& a, const float* sm, int i) {
    constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T, D = C::D;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N;
    const AtomFrame fr = atom_frame(a, i);
    const int ti = fr.ti;
    const float rcR2 = a.rc_rad * a.rc_rad, rcA2 = a.rc_ang * a.rc_ang;
    const float irR = 1.0f / a.rc_rad, irA = 1.0f / a.rc_ang;

    // radial: species-resolved basis sums F[t][k] = sum_{j of species t} Q_k(r_ij)
    float fb[T][KR];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < KR; ++k) fb[t][k] = 0.0f;
    const int cnt = a.cnt[i], cnt_ang = a.cnt_ang[i];
    int nc = 0, ncr = 0;
    // software pipeline: neighbour index two slots ahead, its position one ahead
    int j_nx = cnt > 0 ? a.nbr[i] : 0;
    int j_nx2 = cnt > 1 ? a.nbr[N + i] : 0;
    float4 p_nx = a.pos4[j_nx];
    int sh_nx = (!MINIMG && cnt > 0) ? a.shift[i] : 0;
    for (int s = 0; s < cnt; ++s) {
        const int j = j_nx;
        const float4 pj = p_nx;
        const int sh = sh_nx;
        if (s + 1 < cnt) {
            j_nx = j_nx2;
            p_nx = a.pos4[j_nx];
            if (!MINIMG) sh_nx = a.shift[(s + 1) * N + i];
            if (s + 2 < cnt) j_nx2 = a.nbr[(s + 2) * N + i];
        }
        float dx, dy, dz;
        pair_vector(fr.pi, pj, fr.Lx, fr.Ly, fr.Lz, fr.iLx, fr.iLy, fr.iLz, MINIMG, sh, dx, dy, dz);
        const float d2 = dist2(dx, dy, dz);
        const int tj = f2i(pj.w);
        if (d2 < rcR2) {
            a.compr[ncr * N + i] = make_float4(dx, dy, dz, i2f((int)(((unsigned)j << 2) | (unsigned)tj)));
            ++ncr;
            float f[KR];
            basis<KR>(sqrt_f(d2), irR, f);
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float w = (tj == t) ? 1.0f : 0.0f;
#pragma unroll
                for (int k = 0; k < KR; ++k) fb[t][k] = fmaf(w, f[k], fb[t][k]);
            }
        }
        if (s < cnt_ang) {
            const int addr = a.rev[s * N + i] * N + j;
            if (d2 < rcA2) {
                a.comp[nc * N + i] =
                    make_float4(dx, dy, dz, i2f((int)(((unsigned)addr << 2) | (unsigned)tj)));
                ++nc;
            } else {
                a.fin[addr] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
        }
    }
    a.cnt_comp[i] = nc;
    a.cnt_compr[i] = ncr;

    float q[D];
#pragma unroll
    for (int n = 0; n < NR; ++n) {
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < T; ++t) {
            const float* c = sm + sl.cR + (ti * T + t) * C::SR + n * KR;
#pragma unroll
            for (int k = 0; k < KR; ++k) acc = fmaf(c[k], fb[t][k], acc);
        }
        q[n] = acc;
        NEP_SCHED_BARRIER();
    }
    if (a.fb_out) {
#pragma unroll
        for (int t = 0; t < T; ++t)
#pragma unroll
            for (int k = 0; k < KR; ++k) a.fb_out[(t * KR + k) * N + i] = fb[t][k];
    }

    // angular: S_nlm = sum_j g_n(r_ij) P_lm(rhat_ij)
    float S[NA][kLM];
#pragma unroll
    for (int n = 0; n < NA; ++n)
#pragma unroll
        for (int m = 0; m < kLM; ++m) S[n][m] = 0.0f;
    float4 e_nx = nc > 0 ? a.comp[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int c = 0; c < nc; ++c) {
        const float4 e = e_nx;
        if (c + 1 < nc) e_nx = a.comp[(c + 1) * N + i];
        const int tj = f2i(e.w) & 3;
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        const float ir = rcp_f(r);
        float f[KA];
        basis<KA>(r, irA, f);
        const float* cc = sm + sl.cA + (ti * T + tj) * C::SA;
        float g[NA];
#pragma unroll
        for (int n = 0; n < NA; ++n) {
            float acc = 0.0f;
#pragma unroll
            for (int k = 0; k < KA; ++k) acc = fmaf(cc[n * KA + k], f[k], acc);
            g[n] = acc;
        }
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            float Y, gx, gy, gz;
            harm_m(m, ht, Y, gx, gy, gz);
#pragma unroll
            for (int n = 0; n < NA; ++n) S[n][m] = fmaf(g[n], Y, S[n][m]);
        }
    }
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float ql[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int m = 0; m < kLM; ++m) ql[lm_l(m) - 1] = fmaf(clm(m) * S[n][m], S[n][m], ql[lm_l(m) - 1]);
#pragma unroll
        for (int l = 0; l < 4; ++l) q[NR + n * 4 + l] = ql[l];
        if (C::H4) q[NR + NA * 4 + n] = fourbody(&S[n][3], nullptr);
#pragma unroll
        for (int m = 0; m < kLM; ++m) a.S[(n * kLM + m) * N + i] = S[n][m];
    }

    if (a.q16) {
        // mixed precision: hand q to the tensor-core network as a 16-bit row
        constexpr int Kp = (D + 15) / 16 * 16;
        unsigned* row = reinterpret_cast<unsigned*>(a.q16) + (size_t)i * (Kp / 2);
#pragma unroll
        for (int d = 0; d < Kp; d += 2) {
            const float x0 = d < D ? q[d] : 0.0f, x1 = d + 1 < D ? q[d + 1] : 0.0f;
            unsigned bits;
            if (a.q16_kind == 2) {
                __nv_bfloat162 v = __floats2bfloat162_rn(x0, x1);
                memcpy(&bits, &v, 4);
            } else {
                __half2 v = __floats2half2_rn(x0, x1);
                memcpy(&bits, &v, 4);
            }
            row[d / 2] = bits;
        }
        return;
    }

    // network E_i = sum_h w1 tanh(W0 q + b0) + b1 and p = dE_i/dq
    const float* W0 = sm + sl.W0 + ti * sl.SW;
    const float* b0 = sm + sl.b0 + ti * sl.HS;
    const float* w1 = sm + sl.w1 + ti * sl.HS;
    float E = sm[sl.b1 + ti];
    float p[D];
#pragma unroll
    for (int d = 0; d < D; ++d) p[d] = 0.0f;
    for (int h = 0; h < a.H; ++h) {
        const float* w = W0 + h * D;
        float z = b0[h];
#pragma unroll
        for (int d = 0; d < D; ++d) z = fmaf(w[d], q[d], z);
        const float t = tanh_f(z);
        const float wh = w1[h];
        E = fmaf(wh, t, E);
        const float sg = wh * (1.0f - t * t);
#pragma unroll
        for (int d = 0; d < D; ++d) p[d] = fmaf(sg, w[d], p[d]);
    }
    a.e_atom[i] = E;
#pragma unroll
    for (int d = NR; d < D; ++d) a.pang[(d - NR) * N + i] = p[d];
    if (a.q_out) {
#pragma unroll
        for (int d = 0; d < D; ++d) a.q_out[d * N + i] = q[d];
    }
    if (a.p_out) {
#pragma unroll
        for (int d = 0; d < D; ++d) a.p_out[d * N + i] = p[d];
    }
    // radial adjoint projected on the neighbour species:
    // P[i][t][k] = sum_n dE/dq_n cR[Zi][t][n][k]
#pragma unroll
    for (int t = 0; t < T; ++t) {
        const float* c = sm + sl.cR + (ti * T + t) * C::SR;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            float acc = 0.0f;
#pragma unroll
            for (int n = 0; n < NR; ++n) acc = fmaf(p[n], c[n * KR + k], acc);
            a.Pr[(i * T + t) * KR + k] = acc;
            NEP_SCHED_BARRIER();
        }
    }
}

// ---------------------------------------------------------------------------
// pair forces and per-atom virial, one atom
// ---------------------------------------------------------------------------
template <class C, bool MINIMG>
NEP_HD void force_atom(const EvalArgs& a, const float* sm, int i) {
    constexpr int NR = C::NR, NA = C::NA, KR = C::KR, KA = C::KA, T = C::T;
    (void)NR;
    const SmemLayout sl = smem_layout<C>(a.H);
    const int N = a.N;
    const AtomFrame fr = atom_frame(a, i);
    const int ti = fr.ti;
    const float irR = 1.0f / a.rc_rad, irA = 1.0f / a.rc_ang;

    float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
    float W[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) W[k] = 0.0f;

    // dE_i/dS_nlm = 2 C_lm S_nlm dE/dq_nl (+ the 4-body chain through l = 2)
    float Sb[NA][kLM];
#pragma unroll
    for (int n = 0; n < NA; ++n) {
        float pl[4];
#pragma unroll
        for (int l = 0; l < 4; ++l) pl[l] = a.pang[(n * 4 + l) * N + i];
        float s2[5];
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            const float s = a.S[(n * kLM + m) * N + i];
            if (m >= 3 && m < 8) s2[m - 3] = s;
            Sb[n][m] = 2.0f * clm(m) * pl[lm_l(m) - 1] * s;
        }
        if (C::H4) {
            const float p4 = a.pang[(NA * 4 + n) * N + i];
            float ds[5];
            fourbody(s2, ds);
#pragma unroll
            for (int m = 0; m < 5; ++m) Sb[n][3 + m] = fmaf(p4, ds[m], Sb[n][3 + m]);
        }
    }

    // angular pairs (compacted by desc): owner-side force, scattered to the
    // reverse slot for the gather of F_j
    const int nc = a.cnt_comp[i];
    float4 e_nx = nc > 0 ? a.comp[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int c = 0; c < nc; ++c) {
        const float4 e = e_nx;
        if (c + 1 < nc) e_nx = a.comp[(c + 1) * N + i];
        const int bits = f2i(e.w);
        const int tj = bits & 3;
        const int addr = (int)((unsigned)bits >> 2);
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        const float ir = rcp_f(r);
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
                    const float cv = cc[n * KA + k];
                    u = fmaf(cv, f[k], u);
                    v = fmaf(cv, fp[k], v);
                }
                g[n] = u;
                gp[n] = v;
            }
        }
        const HarmTerms ht = harm_terms(e.x * ir, e.y * ir, e.z * ir);
        // f_ij = u sum_m (b_m - l a_m / r) Y_m + (1/r) sum_m a_m grad P_m(u),
        // a_m = sum_n Sb[n][m] g_n, b_m = sum_n Sb[n][m] g'_n
        float rad = 0.0f, Gx = 0.0f, Gy = 0.0f, Gz = 0.0f;
#pragma unroll
        for (int m = 0; m < kLM; ++m) {
            float am = 0.0f, bm = 0.0f;
#pragma unroll
            for (int n = 0; n < NA; ++n) {
                am = fmaf(Sb[n][m], g[n], am);
                bm = fmaf(Sb[n][m], gp[n], bm);
            }
            float Y, hx, hy, hz;
            harm_m(m, ht, Y, hx, hy, hz);
            rad = fmaf(fmaf(-(float)lm_l(m) * ir, am, bm), Y, rad);
            Gx = fmaf(am, hx, Gx);
            Gy = fmaf(am, hy, Gy);
            Gz = fmaf(am, hz, Gz);
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

    // radial pairs: dE_i/dr_ij + dE_j/dr_ij along rhat, computed from the
    // species-projected adjoints P of both atoms
    float Pi[T][KR];
#pragma unroll
    for (int t = 0; t < T; ++t)
#pragma unroll
        for (int k = 0; k < KR; ++k) Pi[t][k] = a.Pr[(i * T + t) * KR + k];
    // compacted radial pairs (all inside rc_rad): no divergence on the cutoff
    float Wr[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};   // xx yy zz xy xz yz
    const int ncr = a.cnt_compr[i];
    float4 q_nx = ncr > 0 ? a.compr[i] : make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    for (int s = 0; s < ncr; ++s) {
        const float4 e = q_nx;
        if (s + 1 < ncr) q_nx = a.compr[(s + 1) * N + i];
        const int bits = f2i(e.w);
        const int tj = bits & 3;
        const int j = (int)((unsigned)bits >> 2);
        const float4* Pj4 = reinterpret_cast<const float4*>(a.Pr + (j * T + ti) * KR);
        const float r = sqrt_f(dist2(e.x, e.y, e.z));
        const float ir = rcp_f(r);
        float f[KR], fp[KR];
        basis_d<KR>(r, irR, f, fp);
        float dEi = 0.0f, dEj = 0.0f;
#pragma unroll
        for (int k4 = 0; k4 < KR / 4; ++k4) {
            const float4 pj = Pj4[k4];
            dEj = fmaf(pj.x, fp[4 * k4 + 0], dEj);
            dEj = fmaf(pj.y, fp[4 * k4 + 1], dEj);
            dEj = fmaf(pj.z, fp[4 * k4 + 2], dEj);
            dEj = fmaf(pj.w, fp[4 * k4 + 3], dEj);
        }
#pragma unroll
        for (int k = (KR / 4) * 4; k < KR; ++k) dEj = fmaf(a.Pr[(j * T + ti) * KR + k], fp[k], dEj);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            float pk = Pi[0][k];
#pragma unroll
            for (int t = 1; t < T; ++t) pk = (tj == t) ? Pi[t][k] : pk;
            dEi = fmaf(pk, fp[k], dEi);
        }
        const float tot = (dEi + dEj) * ir;
        Fx = fmaf(tot, e.x, Fx); Fy = fmaf(tot, e.y, Fy); Fz = fmaf(tot, e.z, Fz);
        // W -= f_ij (x) r_ij with f_ij = dE_i/dr rhat: symmetric part only
        const float w = dEi * ir;
        const float wx = w * e.x, wy = w * e.y, wz = w * e.z;
        Wr[0] = fmaf(wx, e.x, Wr[0]); Wr[1] = fmaf(wy, e.y, Wr[1]); Wr[2] = fmaf(wz, e.z, Wr[2]);
        Wr[3] = fmaf(wx, e.y, Wr[3]); Wr[4] = fmaf(wx, e.z, Wr[4]); Wr[5] = fmaf(wy, e.z, Wr[5]);
    }
    W[0] -= Wr[0]; W[4] -= Wr[1]; W[8] -= Wr[2];
    W[1] -= Wr[3]; W[3] -= Wr[3];
    W[2] -= Wr[4]; W[6] -= Wr[4];
    W[5] -= Wr[5]; W[7] -= Wr[5];
    a.fpart[i] = Fx;
    a.fpart[N + i] = Fy;
    a.fpart[2 * N + i] = Fz;
#pragma unroll
    for (int k = 0; k < 9; ++k) a.wat[k * N + i] = W[k];
}

// ---------------------------------------------------------------------------
// kernels and launchers
// ---------------------------------------------------------------------------
#if defined(__CUDACC__)
// Resident blocks per SM that the register allocation is sized for
// (65536 / (128 x MINB) registers per thread: 255, 168 or 128).  Each kernel
// is compiled for MINB = 2, 3 and 4; the runtime picks one per system size
// class (nep_autotune), by default 3 for the descriptor kernel and 2 for the
// force kernel, which keeps dE/dS (n_ang x 24 floats) in registers.
NEP_HD constexpr int variant_minb(int v) { return v + 2; }

template <class C, bool MINIMG, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_desc(const EvalArgs a) {
    extern __shared__ float sm[];
    load_model<C>(sm, a.params, a.H, threadIdx.x, blockDim.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N) desc_atom<C, MINIMG>(a, sm, i);
}

template <class C, bool MINIMG, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_force(const EvalArgs a) {
    extern __shared__ float sm[];
    load_model<C>(sm, a.params, a.H, threadIdx.x, blockDim.x);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < a.N) force_atom<C, MINIMG>(a, sm, i);
}

template <class C>
size_t smem_bytes_of(int H) { return sizeof(float) * (size_t)smem_layout<C>(H).total; }

template <class C, int MINB>
void launch_desc_v(const EvalArgs& a, cudaStream_t st, size_t smem, int grid) {
    if (a.min_image)
        k_desc<C, true, MINB><<<grid, kBlock, smem, st>>>(a);
    else
        k_desc<C, false, MINB><<<grid, kBlock, smem, st>>>(a);
}
template <class C, int MINB>
void launch_force_v(const EvalArgs& a, cudaStream_t st, size_t smem, int grid) {
    if (a.min_image)
        k_force<C, true, MINB><<<grid, kBlock, smem, st>>>(a);
    else
        k_force<C, false, MINB><<<grid, kBlock, smem, st>>>(a);
}

template <class C>
cudaError_t launch_desc_t(const EvalArgs& a, cudaStream_t st, int v) {
    const size_t smem = smem_bytes_of<C>(a.H);
    const int grid = (a.N + kBlock - 1) / kBlock;
    if (grid == 0) return cudaSuccess;
    if (v == 0) launch_desc_v<C, 2>(a, st, smem, grid);
    else if (v == 2) launch_desc_v<C, 4>(a, st, smem, grid);
    else launch_desc_v<C, 3>(a, st, smem, grid);
    return cudaGetLastError();
}

template <class C>
cudaError_t launch_force_t(const EvalArgs& a, cudaStream_t st, int v) {
    const size_t smem = smem_bytes_of<C>(a.H);
    const int grid = (a.N + kBlock - 1) / kBlock;
    if (grid == 0) return cudaSuccess;
    if (v == 1) launch_force_v<C, 3>(a, st, smem, grid);
    else if (v == 2) launch_force_v<C, 4>(a, st, smem, grid);
    else launch_force_v<C, 2>(a, st, smem, grid);
    return cudaGetLastError();
}

template <class C, int MINB>
cudaError_t init_v(int smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_desc<C, true, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(k_desc<C, false, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    if ((e = cudaFuncSetAttribute(k_force<C, true, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    return cudaFuncSetAttribute(k_force<C, false, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <class C>
cudaError_t init_t(int H) {
    const int smem = (int)smem_bytes_of<C>(H);
    cudaError_t e;
    if ((e = init_v<C, 2>(smem))) return e;
    if ((e = init_v<C, 3>(smem))) return e;
    return init_v<C, 4>(smem);
}

#define NEP_DEFINE_KERNEL_SET(NAME, NR, NA, KR, KA, H4, T)                                    \
    extern const KernelSet NAME = {NR, NA, KR, KA, H4, T,                                        \
                                   &smem_bytes_of<Cfg<NR, NA, KR, KA, H4, T>>,                   \
                                   &init_t<Cfg<NR, NA, KR, KA, H4, T>>,                          \
                                   &launch_desc_t<Cfg<NR, NA, KR, KA, H4, T>>,                   \
                                   &launch_force_t<Cfg<NR, NA, KR, KA, H4, T>>,                  \
                                   &launch_mlp_tc_t<Cfg<NR, NA, KR, KA, H4, T>>,                 \
                                   &train_init_t<Cfg<NR, NA, KR, KA, H4, T>>,                    \
                                   &train_t<Cfg<NR, NA, KR, KA, H4, T>>,                         \
                                   &grad_chunks_t<Cfg<NR, NA, KR, KA, H4, T>>};
#endif

}  // namespace nep
