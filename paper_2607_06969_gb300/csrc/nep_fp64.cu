// FP64 evaluation of energies, forces and virial, and the FP64 training
// gradient.
//
// The operators of Section 3.2 run in float64 as well as float32.  This path
// computes Eqs. 1-4 and 11-21 with every intermediate in double: positions
// (FP32 inputs) are promoted, the parameters are FP64, and pairs are kept by
// r < rc in double.  Hyper-parameters are runtime values.  G lanes per atom
// split its neighbour list: G = 1 once N fills the GPU, up to a warp for a
// few hundred atoms, so that small systems still reach every SM.
//
// Evaluation, two passes over the list:
//   k64_atom  : the species-resolved radial basis sums F[t][k] and q_n
//               (Eq. 11), S_nlm and q_nl (Eqs. 16-17), q4_n, the network
//               (Eq. 2), E_i, dE_i/dq_n (radial) and R_nlm = dE_i/dS_nlm
//   k64_force : F_i = sum_j [dE_i/dr_ij - dE_j/dr_ji] (Eq. 3), each pair
//               derivative recomputed from its owner's dE/dq and R; per-atom
//               virial W_i = -sum_j dE_i/dr_ij (x) r_ij (Eq. 4)
// then FP64 sums per 1,024-atom chunk and per configuration in a fixed order.
//
// Training gradient: the gradient of Phi = sum_b aE_b E_b + sum_i lam_i . F_i
// + sum_b mu_b : V_b at fixed adjoints (the loss gradient of Eqs. 18-21 when
// they are the loss adjoints).  With dr_ij = -(lam_j - lam_i) - mu r_ij,
// Phi = sum_i [aE E_i + p_i . dq_i], p = dE/dq, dq the tangent of q along dr.
//   k64_grad_atom : descriptors and network again, the tangent dq (radial
//                   DF[t][k] = sum_j Q'_k (rhat . dr), angular dS_nlm), the
//                   network's second-order terms (alpha, beta, gamma,
//                   rho = aE p + d(p . dq)/dq), P = dPhi/dS, R = dPhi/d(dS),
//                   and per angular pair X_n = sum_m P_nm Y_m + R_nm dY_m . dr,
//                   Z_n = (rhat . dr) sum_m R_nm Y_m, summed into
//                   bins[t][n][k] = sum_{j of t} Q_k X_n + Q'_k Z_n; the
//                   per-atom factors of every parameter's gradient are staged
//   k64_grad_partial / k64_grad_final : per 1,024-atom chunk, each parameter
//                   summed over the chunk's atoms of its species; then the
//                   chunks in order
//
// Lane partials are combined by an xor butterfly, whose fixed tree leaves
// the same bits in every lane of the group; every pair term is evaluated by
// both of its atoms, so nothing is scattered, and for a given N (which fixes
// G) every result is deterministic.
#include <cuda_runtime.h>

#include "nep_device.cuh"
#include "nep_internal.h"

namespace nep {
namespace {

constexpr int kF64Block = 128;
constexpr int kF64MaxD = kF64MaxN * 6;              // n_rad + 5 n_ang
constexpr int kF64MaxTK = kMaxTypes * kF64MaxK;     // n_types * k_rad
constexpr double kPi = 3.141592653589793;

// The evaluation below is written once for two argument types: F64Args (every
// intermediate in double) and F32Args (the generic FP32 evaluation, any
// hyper-parameters within the same bounds).  R is the argument type's scalar.
template <class A>
struct ScalarOf;
template <>
struct ScalarOf<F64Args> {
    using type = double;
};
template <>
struct ScalarOf<F32Args> {
    using type = float;
};
template <class A>
using ScalarT = typename ScalarOf<A>::type;

__device__ __forceinline__ void sincospi_r(double z, double* s, double* c) { sincospi(z, s, c); }
__device__ __forceinline__ void sincospi_r(float z, float* s, float* c) { sincospif(z, s, c); }
__device__ __forceinline__ double tanh_r(double x) { return tanh(x); }
__device__ __forceinline__ float tanh_r(float x) { return tanhf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double rint_r(double x) { return rint(x); }
__device__ __forceinline__ float rint_r(float x) { return rintf(x); }

// Q_k(r) and dQ_k/dr for k < K at r < rc: Q_k = (T_k(x) + 1)/2 f_c(r),
// x = 2(r/rc - 1)^2 - 1, f_c = (1 + cos(pi r/rc))/2 (Eqs. 12-15)
template <class R>
__device__ void basis64(R r, R rc, int K, R* f, R* fp) {
    const R z = r / rc;
    R sp, cp;
    sincospi_r(z, &sp, &cp);
    const R fc2 = R(0.25) * (R(1.0) + cp);                 // f_c / 2
    const R dfc2 = R(-0.25) * R(kPi) / rc * sp;            // (d f_c/dr) / 2
    const R t = z - R(1.0), x = R(2.0) * t * t - R(1.0), dx = R(4.0) * t / rc;
    R Tm = R(1.0), Tk = x, dTm = R(0.0), dTk = R(1.0);
    f[0] = R(2.0) * fc2;
    fp[0] = R(2.0) * dfc2;
    if (K > 1) {
        f[1] = (x + R(1.0)) * fc2;
        fp[1] = dx * fc2 + (x + R(1.0)) * dfc2;
    }
    for (int k = 2; k < K; ++k) {
        const R Tn = R(2.0) * x * Tk - Tm;
        const R dTn = R(2.0) * Tk + R(2.0) * x * dTk - dTm;
        f[k] = (Tn + R(1.0)) * fc2;
        fp[k] = dTn * dx * fc2 + (Tn + R(1.0)) * dfc2;
        Tm = Tk; Tk = Tn; dTm = dTk; dTk = dTn;
    }
}

// sum over the G aligned lanes of an atom; every lane receives the same bits.
// The shuffles name only the group's lanes: a group whose atom index is past
// N leaves as a whole, while the other groups of its warp go on.
template <int G, class R>
__device__ __forceinline__ R group_sum(R v) {
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

template <class R>
struct FrameT {
    int i, ti, b;
    R L[3], x, y, z;
};
using Frame64 = FrameT<double>;
template <class A>
__device__ FrameT<ScalarT<A>> frame64(const A& a, int i) {
    FrameT<ScalarT<A>> fr;
    fr.i = i;
    fr.ti = a.type[i];
    fr.b = a.cfg[i];
    for (int c = 0; c < 3; ++c) fr.L[c] = a.box[3 * fr.b + c];
    fr.x = a.pos[i];
    fr.y = a.pos[a.N + i];
    fr.z = a.pos[2 * a.N + i];
    return fr;
}

// list slot s of atom fr.i: r_ij = (r_j - r_i) + s L in R, with the list's
// image or the minimum image; false when r >= rc_rad
template <class R>
struct PairT {
    int j, tj;
    R d[3], r, u[3];
};
using Pair64 = PairT<double>;
template <class A, class R>
__device__ bool pair_at(const A& a, const FrameT<R>& fr, int s, PairT<R>& p) {
    const int N = a.N;
    p.j = a.nbr[(size_t)s * N + fr.i];
    const R ux = (R)a.pos[p.j] - fr.x, uy = (R)a.pos[N + p.j] - fr.y, uz = (R)a.pos[2 * N + p.j] - fr.z;
    R sx, sy, sz;
    if (a.shift) {
        int ix, iy, iz;
        unpack_shift(a.shift[(size_t)s * N + fr.i], ix, iy, iz);
        sx = (R)ix; sy = (R)iy; sz = (R)iz;
    } else {
        sx = -rint_r(ux / fr.L[0]);
        sy = -rint_r(uy / fr.L[1]);
        sz = -rint_r(uz / fr.L[2]);
    }
    p.d[0] = ux + sx * fr.L[0];
    p.d[1] = uy + sy * fr.L[1];
    p.d[2] = uz + sz * fr.L[2];
    p.r = sqrt_r(p.d[0] * p.d[0] + p.d[1] * p.d[1] + p.d[2] * p.d[2]);
    if (!(p.r < a.rc_rad)) return false;
    p.tj = a.type[p.j];
    const R ir = R(1.0) / p.r;
    for (int c = 0; c < 3; ++c) p.u[c] = p.d[c] * ir;
    return true;
}

// g_n = sum_k cA[ti][tj][n][k] Q_k (and g'_n with Q'_k)
template <class A, class R>
__device__ void angular_g(const A& a, int ti, int tj, const R* f, const R* fp, R* g, R* gp) {
    const R* cA = a.prm + a.L.off_cA + (size_t)(ti * a.T + tj) * a.NA * a.KA;
    for (int n = 0; n < a.NA; ++n) {
        R u = R(0.0), v = R(0.0);
        for (int k = 0; k < a.KA; ++k) {
            u += cA[n * a.KA + k] * f[k];
            v += cA[n * a.KA + k] * fp[k];
        }
        g[n] = u;
        gp[n] = v;
    }
}

// g_n only (the descriptors need no derivative)
template <class A, class R>
__device__ void angular_g_value(const A& a, int ti, int tj, const R* f, R* g) {
    const R* cA = a.prm + a.L.off_cA + (size_t)(ti * a.T + tj) * a.NA * a.KA;
    for (int n = 0; n < a.NA; ++n) {
        R u = R(0.0);
        for (int k = 0; k < a.KA; ++k) u += cA[n * a.KA + k] * f[k];
        g[n] = u;
    }
}

// q [D], S [NA*24] and the species-resolved radial basis sums F [T*KR] of
// atom fr.i (the same values in every lane of its group)
template <int G, class A, class R>
__device__ void descriptors64(const A& a, const FrameT<R>& fr, int lane, R* q, R* S, R* F) {
    const int T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA;
    R f[kF64MaxK], fp[kF64MaxK], g[kF64MaxN];
    for (int x = 0; x < T * KR; ++x) F[x] = R(0.0);
    for (int x = 0; x < NA * kLM; ++x) S[x] = R(0.0);
    const int nc = a.cnt[fr.i];
    for (int s = lane; s < nc; s += G) {
        PairT<R> p;
        if (!pair_at(a, fr, s, p)) continue;
        basis64(p.r, (R)a.rc_rad, KR, f, fp);
        for (int k = 0; k < KR; ++k) F[p.tj * KR + k] += f[k];
        if (!(p.r < a.rc_ang)) continue;
        basis64(p.r, (R)a.rc_ang, KA, f, fp);
        angular_g_value(a, fr.ti, p.tj, f, g);
        const HarmTermsT<R> ht = harm_terms(p.u[0], p.u[1], p.u[2]);
        for (int m = 0; m < kLM; ++m) {
            R Y, gx, gy, gz;
            harm_m(m, ht, Y, gx, gy, gz);
            for (int n = 0; n < NA; ++n) S[n * kLM + m] += g[n] * Y;
        }
    }
    for (int x = 0; x < T * KR; ++x) F[x] = group_sum<G>(F[x]);
    for (int x = 0; x < NA * kLM; ++x) S[x] = group_sum<G>(S[x]);
    // q_n = sum_t sum_k cR[ti][t][n][k] F[t][k]
    const R* cR = a.prm + a.L.off_cR + (size_t)fr.ti * T * NR * KR;
    for (int n = 0; n < NR; ++n) {
        R v = R(0.0);
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < KR; ++k) v += cR[(t * NR + n) * KR + k] * F[t * KR + k];
        q[n] = v;
    }
    // q_nl = sum_m C_lm S_nlm^2 and q4_n = tr(A_n^3)
    for (int n = 0; n < NA; ++n) {
        for (int l = 0; l < 4; ++l) q[NR + n * 4 + l] = R(0.0);
        for (int m = 0; m < kLM; ++m) {
            const R v = S[n * kLM + m];
            q[NR + n * 4 + lm_l(m) - 1] += (R)clm(m) * v * v;
        }
        if (a.H4) q[NR + NA * 4 + n] = fourbody<R>(S + n * kLM + 3, nullptr);
    }
}

__global__ void k_promote(const float* src, double* dst, int n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) dst[x] = (double)src[x];
}

// ------------------------------------------------------------ evaluation
// A warp's groups all belong to one block row; G divides 32 and kF64Block,
// so no group straddles a warp.
template <int G, class A>
__global__ void __launch_bounds__(kF64Block) k64_atom(const A a) {
    using R = ScalarT<A>;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    if (i >= a.N) return;
    const int N = a.N, NR = a.NR, NA = a.NA, H = a.H, D = a.D;
    const FrameT<R> fr = frame64(a, i);
    R q[kF64MaxD], S[kF64MaxN * kLM], F[kF64MaxTK];
    descriptors64<G>(a, fr, lane, q, S, F);
    // network: E_i = w1 . tanh(W0 q + b0) + b1, dE/dq = W0^T (w1 (1 - t^2));
    // lane takes hidden units h = lane, lane + G, ...
    const R* W0 = a.prm + (size_t)fr.ti * a.L.mlp_stride;
    const R* b0 = W0 + (size_t)H * D;
    const R* w1 = b0 + H;
    R E = R(0.0), pq[kF64MaxD];
    for (int d = 0; d < D; ++d) pq[d] = R(0.0);
    for (int h = lane; h < H; h += G) {
        const R* w = W0 + (size_t)h * D;
        R z = b0[h];
        for (int d = 0; d < D; ++d) z += w[d] * q[d];
        const R th = tanh_r(z);
        E += w1[h] * th;
        const R c = w1[h] * (R(1.0) - th * th);
        for (int d = 0; d < D; ++d) pq[d] += c * w[d];
    }
    E = group_sum<G>(E) + w1[H];
    for (int d = 0; d < D; ++d) pq[d] = group_sum<G>(pq[d]);
    if (lane == 0) a.e[i] = E;
    for (int n = lane; n < NR; n += G) a.p[(size_t)n * N + i] = pq[n];
    // R_nlm = dE/dq_nl 2 C_lm S_nlm (+ dE/dq4_n dq4_n/dS_n2m), entries split over lanes
    for (int x = lane; x < NA * kLM; x += G) {
        const int n = x / kLM, m = x % kLM;
        R v = R(2.0) * (R)clm(m) * pq[NR + n * 4 + lm_l(m) - 1] * S[x];
        if (a.H4 && m >= 3 && m < 8) {
            R J[5];
            fourbody<R>(S + n * kLM + 3, J);
            v += pq[NR + NA * 4 + n] * J[m - 3];
        }
        a.R[(size_t)x * N + i] = v;
    }
}

// dE_o/dr_oj for owner o of species to, neighbour species tn, distance r and
// unit vector u = r_oj / r
template <class A, class R>
__device__ void pair_deriv(const A& a, int o, int to, int tn, R r, const R* u, R* fo) {
    const int N = a.N, T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA;
    R f[kF64MaxK], fp[kF64MaxK], g[kF64MaxN], gp[kF64MaxN];
    basis64(r, (R)a.rc_rad, KR, f, fp);
    const R* cR = a.prm + a.L.off_cR + (size_t)(to * T + tn) * NR * KR;
    R gr = R(0.0);
    for (int n = 0; n < NR; ++n) {
        R dg = R(0.0);
        for (int k = 0; k < KR; ++k) dg += cR[n * KR + k] * fp[k];
        gr += a.p[(size_t)n * N + o] * dg;
    }
    fo[0] = gr * u[0];
    fo[1] = gr * u[1];
    fo[2] = gr * u[2];
    if (!(r < a.rc_ang)) return;
    basis64(r, (R)a.rc_ang, KA, f, fp);
    angular_g(a, to, tn, f, fp, g, gp);
    const HarmTermsT<R> ht = harm_terms(u[0], u[1], u[2]);
    R Y[kLM], Gr[kLM][3];
    for (int m = 0; m < kLM; ++m) harm_m(m, ht, Y[m], Gr[m][0], Gr[m][1], Gr[m][2]);
    const R ir = R(1.0) / r;
    for (int n = 0; n < NA; ++n) {
        // d S_nlm / d r_oj = g'_n Y_m u + g_n (grad P_m - l P_m u) / r
        R sY = R(0.0), slY = R(0.0), sg[3] = {R(0.0), R(0.0), R(0.0)};
        for (int m = 0; m < kLM; ++m) {
            const R Rv = a.R[(size_t)(n * kLM + m) * N + o];
            sY += Rv * Y[m];
            slY += Rv * (R)lm_l(m) * Y[m];
            sg[0] += Rv * Gr[m][0];
            sg[1] += Rv * Gr[m][1];
            sg[2] += Rv * Gr[m][2];
        }
        for (int c = 0; c < 3; ++c) fo[c] += gp[n] * sY * u[c] + g[n] * ir * (sg[c] - slY * u[c]);
    }
}

template <int G, class A>
__global__ void __launch_bounds__(kF64Block) k64_force(const A a) {
    using R = ScalarT<A>;
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    if (i >= a.N) return;
    const int N = a.N;
    const FrameT<R> fr = frame64(a, i);
    R F[3] = {R(0.0), R(0.0), R(0.0)}, W[9];
    for (int c = 0; c < 9; ++c) W[c] = R(0.0);
    const int nc = a.cnt[i];
    for (int s = lane; s < nc; s += G) {
        PairT<R> p;
        if (!pair_at(a, fr, s, p)) continue;
        const R v[3] = {-p.u[0], -p.u[1], -p.u[2]};
        R fij[3], fji[3];
        pair_deriv(a, i, fr.ti, p.tj, p.r, p.u, fij);
        pair_deriv(a, p.j, p.tj, fr.ti, p.r, v, fji);
        for (int c = 0; c < 3; ++c) F[c] += fij[c] - fji[c];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) W[3 * x + y] -= fij[x] * p.d[y];
    }
    for (int c = 0; c < 3; ++c) F[c] = group_sum<G>(F[c]);
    for (int c = 0; c < 9; ++c) W[c] = group_sum<G>(W[c]);
    for (int c = lane; c < 3; c += G) a.force[(size_t)c * N + i] = F[c];
    for (int c = lane; c < 9; c += G) a.w[(size_t)c * N + i] = W[c];
}

__device__ int segment_of(const int* off, int B, int x) {
    int lo = 0, hi = B;   // off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// FP64 sums of E_i and W_i per 1,024-atom chunk: strided per-thread sums,
// then warp shuffles and the warp sums in order; atoms from n_owned on are
// left out (the owned prefix of a spatial decomposition's local system)
constexpr int kF64Red = 256;
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < kF64Red / 32; ++q) s += red[q];
    return s;
}

template <class A>
__global__ void __launch_bounds__(kF64Red) k64_chunk_reduce(const A a) {
    const int k = blockIdx.x, B = a.B, N = a.N;
    if (k >= a.chunk_start[B]) return;
    const int b = segment_of(a.chunk_start, B, k);
    const int a0 = a.atom_off[b] + (k - a.chunk_start[b]) * kChunk;
    const int a1 = min(min(a.atom_off[b + 1], a0 + kChunk), a.n_owned);
    double acc[10];
    for (int c = 0; c < 10; ++c) acc[c] = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += kF64Red) {
        acc[0] += (double)a.e[i];
        for (int c = 0; c < 9; ++c) acc[1 + c] += (double)a.w[(size_t)c * N + i];
    }
    __shared__ double red[kF64Red / 32];
    for (int c = 0; c < 10; ++c) {
        const double v = block_sum(acc[c], red);
        if (threadIdx.x == 0) a.partial[(size_t)k * 10 + c] = v;
    }
}

// ------------------------------------------------------------ loss
// Per chunk: the force residual's squared sum and lam_i = dL/dF_i.
__global__ void __launch_bounds__(kF64Red) k64_loss_atoms(const F64Args a, const double* f_lbl, double wF,
                                                         double* lam, double* partial) {
    const int k = blockIdx.x, B = a.B, N = a.N;
    if (k >= a.chunk_start[B]) return;
    const int b = segment_of(a.chunk_start, B, k);
    const int a0 = a.atom_off[b] + (k - a.chunk_start[b]) * kChunk;
    const int a1 = min(a.atom_off[b + 1], a0 + kChunk);
    const double nb = (double)(a.atom_off[b + 1] - a.atom_off[b]);
    const double cf = 2.0 * wF / (3.0 * nb * (double)B);
    double acc = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += kF64Red) {
        for (int c = 0; c < 3; ++c) {
            const double d = a.force[(size_t)c * N + i] - f_lbl[(size_t)c * N + i];
            lam[(size_t)c * N + i] = cf * d;
            acc += d * d;
        }
    }
    __shared__ double red[kF64Red / 32];
    const double v = block_sum(acc, red);
    if (threadIdx.x == 0) partial[k] = v;
}

// Per configuration: the loss terms and the energy and virial adjoints
// (modes as nep_param_grad); the batch loss in a fixed tree.
__global__ void __launch_bounds__(kF64Red) k64_loss_cfg(const F64Args a, const double* partial,
                                                       const double* e_tot, const double* vir,
                                                       const double* e_lbl, const double* v_lbl, double wE,
                                                       double wF, double wV, int mode, double* aE, double* mu,
                                                       double* loss) {
    const int B = a.B;
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += kF64Red) {
        const double nb = (double)(a.atom_off[b + 1] - a.atom_off[b]);
        const double n = nb > 0.0 ? nb : 1.0;
        double sF = 0.0;
        for (int k = a.chunk_start[b]; k < a.chunk_start[b + 1]; ++k) sF += partial[k];
        const double dE = e_tot[b] - e_lbl[b];
        double sV = 0.0;
        for (int c = 0; c < 9; ++c) {
            const double dv = vir[9 * b + c] - v_lbl[9 * b + c];
            sV += dv * dv;
        }
        // mode 0: per-atom normalised energy and virial; mode 1: Eqs. 19-21
        const double nE = mode == 0 ? n * n : n, nV = mode == 0 ? 9.0 * n * n : 9.0 * n;
        const double Lb = wE * dE * dE / nE + wF * sF / (3.0 * n) + wV * sV / nV;
        aE[b] = 2.0 * wE * dE / nE / B;
        for (int c = 0; c < 9; ++c) mu[9 * b + c] = 2.0 * wV * (vir[9 * b + c] - v_lbl[9 * b + c]) / nV / B;
        if (nb > 0.0) acc += Lb;
    }
    __shared__ double red[kF64Red / 32];
    const double v = block_sum(acc, red);
    if (threadIdx.x == 0 && loss) *loss = v / B;
}

// ------------------------------------------------------------ gradient
// Staged per-atom factors, [field][N]: q, dq (D each), alpha, beta, gamma
// (H each), rho and p of the radial n (NR each), F and DF (T KR each), and
// bins (T NA KA).
struct GradFields {
    int q, dq, al, be, ga, rho, p, F, DF, bins, total;
};
__host__ __device__ GradFields grad_fields(const F64Args& a) {
    GradFields g;
    g.q = 0;
    g.dq = g.q + a.D;
    g.al = g.dq + a.D;
    g.be = g.al + a.H;
    g.ga = g.be + a.H;
    g.rho = g.ga + a.H;
    g.p = g.rho + a.NR;
    g.F = g.p + a.NR;
    g.DF = g.F + a.T * a.KR;
    g.bins = g.DF + a.T * a.KR;
    g.total = g.bins + a.T * a.NA * a.KA;
    return g;
}

// dr_ij = -(lam_j - lam_i) - mu r_ij
__device__ void tangent64(const F64Args& a, const double* li, const double* mu, const Pair64& p, double* dr) {
    const int N = a.N;
    for (int c = 0; c < 3; ++c)
        dr[c] = -(a.lam[(size_t)c * N + p.j] - li[c]) -
                (mu[3 * c] * p.d[0] + mu[3 * c + 1] * p.d[1] + mu[3 * c + 2] * p.d[2]);
}

template <int G>
__global__ void __launch_bounds__(kF64Block) k64_grad_atom(const F64Args a) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    if (i >= a.N) return;
    const int N = a.N, T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA, H = a.H, D = a.D;
    const GradFields gf = grad_fields(a);
    const Frame64 fr = frame64(a, i);
    double q[kF64MaxD], S[kF64MaxN * kLM], F[kF64MaxTK];
    descriptors64<G>(a, fr, lane, q, S, F);
    const double li[3] = {a.lam[i], a.lam[N + i], a.lam[2 * N + i]};
    const double* mu = a.mu + 9 * fr.b;
    const double aE = a.aE[fr.b];
    double f[kF64MaxK], fp[kF64MaxK], g[kF64MaxN], gp[kF64MaxN];

    // tangent along dr: DF[t][k] = sum_{j of t} Q'_k (rhat . dr) and
    // dS_nlm = sum_j [g'_n (rhat . dr) Y_m + g_n (grad P_m . dr - l Y_m rhat . dr) / r]
    double DF[kF64MaxTK], dS[kF64MaxN * kLM];
    for (int x = 0; x < T * KR; ++x) DF[x] = 0.0;
    for (int x = 0; x < NA * kLM; ++x) dS[x] = 0.0;
    const int nc = a.cnt[i];
    for (int s = lane; s < nc; s += G) {
        Pair64 p;
        if (!pair_at(a, fr, s, p)) continue;
        double dr[3];
        tangent64(a, li, mu, p, dr);
        const double udr = p.u[0] * dr[0] + p.u[1] * dr[1] + p.u[2] * dr[2];
        basis64(p.r, a.rc_rad, KR, f, fp);
        for (int k = 0; k < KR; ++k) DF[p.tj * KR + k] += fp[k] * udr;
        if (!(p.r < a.rc_ang)) continue;
        basis64(p.r, a.rc_ang, KA, f, fp);
        angular_g(a, fr.ti, p.tj, f, fp, g, gp);
        const HarmTermsT<double> ht = harm_terms(p.u[0], p.u[1], p.u[2]);
        const double ir = 1.0 / p.r;
        for (int m = 0; m < kLM; ++m) {
            double Y, gx, gy, gz;
            harm_m(m, ht, Y, gx, gy, gz);
            const double dY = (gx * dr[0] + gy * dr[1] + gz * dr[2] - lm_l(m) * Y * udr) * ir;
            for (int n = 0; n < NA; ++n) dS[n * kLM + m] += gp[n] * udr * Y + g[n] * dY;
        }
    }
    for (int x = 0; x < T * KR; ++x) DF[x] = group_sum<G>(DF[x]);
    for (int x = 0; x < NA * kLM; ++x) dS[x] = group_sum<G>(dS[x]);
    // dq: radial from DF, angular from S and dS
    double dq[kF64MaxD];
    const double* cR = a.prm + a.L.off_cR + (size_t)fr.ti * T * NR * KR;
    for (int n = 0; n < NR; ++n) {
        double v = 0.0;
        for (int t = 0; t < T; ++t)
            for (int k = 0; k < KR; ++k) v += cR[(t * NR + n) * KR + k] * DF[t * KR + k];
        dq[n] = v;
    }
    for (int n = 0; n < NA; ++n) {
        for (int l = 0; l < 4; ++l) dq[NR + n * 4 + l] = 0.0;
        for (int m = 0; m < kLM; ++m)
            dq[NR + n * 4 + lm_l(m) - 1] += 2.0 * (double)clm(m) * S[n * kLM + m] * dS[n * kLM + m];
        if (a.H4) {
            double J[5];
            fourbody<double>(S + n * kLM + 3, J);
            double v = 0.0;
            for (int m = 0; m < 5; ++m) v += J[m] * dS[n * kLM + 3 + m];
            dq[NR + NA * 4 + n] = v;
        }
    }
    // network and its second-order terms, lane takes h = lane, lane + G, ...:
    // u = W0 dq, alpha = aE w1 s - 2 w1 u t s (coefficient of q in dW0, and
    // db0), beta = w1 s (coefficient of dq), gamma = aE t + s u (dw1);
    // p = W0^T (w1 s), p2 = W0^T (-2 w1 u t s), rho = aE p + p2
    const double* W0 = a.prm + (size_t)fr.ti * a.L.mlp_stride;
    const double* b0 = W0 + (size_t)H * D;
    const double* w1 = b0 + H;
    double pq[kF64MaxD], rho[kF64MaxD];
    for (int d = 0; d < D; ++d) pq[d] = rho[d] = 0.0;
    for (int h = lane; h < H; h += G) {
        const double* w = W0 + (size_t)h * D;
        double z = b0[h], u = 0.0;
        for (int d = 0; d < D; ++d) {
            z += w[d] * q[d];
            u += w[d] * dq[d];
        }
        const double t = tanh(z), sd = 1.0 - t * t, wh = w1[h];
        const double c2 = -2.0 * wh * u * t * sd;
        a.st[(size_t)(gf.al + h) * N + i] = aE * wh * sd + c2;
        a.st[(size_t)(gf.be + h) * N + i] = wh * sd;
        a.st[(size_t)(gf.ga + h) * N + i] = aE * t + sd * u;
        for (int d = 0; d < D; ++d) {
            pq[d] += wh * sd * w[d];
            rho[d] += c2 * w[d];
        }
    }
    for (int d = 0; d < D; ++d) {
        pq[d] = group_sum<G>(pq[d]);
        rho[d] = aE * pq[d] + group_sum<G>(rho[d]);
    }
    // P = dPhi/dS (into dS) and R = dPhi/d(dS) (into S):
    // P_nm = 2 C_lm (rho_nl S_nm + p_nl dS_nm) (+ rho4 J_m + p4 dJ_m),
    // R_nm = 2 C_lm p_nl S_nm (+ p4 J_m)
    for (int n = 0; n < NA; ++n) {
        double J[5] = {0.0, 0.0, 0.0, 0.0, 0.0}, dJ[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        if (a.H4) fourbody_jvp<double>(S + n * kLM + 3, dS + n * kLM + 3, J, dJ);
        const double r4 = a.H4 ? rho[NR + NA * 4 + n] : 0.0, p4 = a.H4 ? pq[NR + NA * 4 + n] : 0.0;
        for (int m = 0; m < kLM; ++m) {
            const int l = lm_l(m) - 1;
            const double c = 2.0 * (double)clm(m), Sv = S[n * kLM + m], dSv = dS[n * kLM + m];
            double Pv = c * (rho[NR + n * 4 + l] * Sv + pq[NR + n * 4 + l] * dSv);
            double Rv = c * pq[NR + n * 4 + l] * Sv;
            if (m >= 3 && m < 8) {
                Pv += r4 * J[m - 3] + p4 * dJ[m - 3];
                Rv += p4 * J[m - 3];
            }
            dS[n * kLM + m] = Pv;
            S[n * kLM + m] = Rv;
        }
    }
    const double* P = dS;
    const double* R = S;
    // bins[t][n][k] = sum_{j of t} Q_k X_n + Q'_k Z_n over the angular pairs
    double bins[kF64MaxBins];
    for (int x = 0; x < T * NA * KA; ++x) bins[x] = 0.0;
    for (int s = lane; s < nc; s += G) {
        Pair64 p;
        if (!pair_at(a, fr, s, p) || !(p.r < a.rc_ang)) continue;
        double dr[3];
        tangent64(a, li, mu, p, dr);
        const double udr = p.u[0] * dr[0] + p.u[1] * dr[1] + p.u[2] * dr[2];
        basis64(p.r, a.rc_ang, KA, f, fp);
        const HarmTermsT<double> ht = harm_terms(p.u[0], p.u[1], p.u[2]);
        const double ir = 1.0 / p.r;
        double X[kF64MaxN], Z[kF64MaxN];
        for (int n = 0; n < NA; ++n) X[n] = Z[n] = 0.0;
        for (int m = 0; m < kLM; ++m) {
            double Y, gx, gy, gz;
            harm_m(m, ht, Y, gx, gy, gz);
            const double dY = (gx * dr[0] + gy * dr[1] + gz * dr[2] - lm_l(m) * Y * udr) * ir;
            for (int n = 0; n < NA; ++n) {
                X[n] += P[n * kLM + m] * Y + R[n * kLM + m] * dY;
                Z[n] += R[n * kLM + m] * Y;
            }
        }
        for (int n = 0; n < NA; ++n)
            for (int k = 0; k < KA; ++k) bins[(p.tj * NA + n) * KA + k] += f[k] * X[n] + fp[k] * udr * Z[n];
    }
    for (int x = 0; x < T * NA * KA; ++x) bins[x] = group_sum<G>(bins[x]);
    // stage the factors, entries split over the lanes
    for (int d = lane; d < D; d += G) {
        a.st[(size_t)(gf.q + d) * N + i] = q[d];
        a.st[(size_t)(gf.dq + d) * N + i] = dq[d];
    }
    for (int n = lane; n < NR; n += G) {
        a.st[(size_t)(gf.rho + n) * N + i] = rho[n];
        a.st[(size_t)(gf.p + n) * N + i] = pq[n];
    }
    for (int x = lane; x < T * KR; x += G) {
        a.st[(size_t)(gf.F + x) * N + i] = F[x];
        a.st[(size_t)(gf.DF + x) * N + i] = DF[x];
    }
    for (int x = lane; x < T * NA * KA; x += G) a.st[(size_t)(gf.bins + x) * N + i] = bins[x];
}

// Each parameter's gradient over one 1,024-atom chunk: the sum, over the
// chunk's atoms of the parameter's species, of a1 b1 + a2 b2 (staged
// factors; b = 1 where absent; aE for a1 of b1).  One warp per parameter,
// lanes over consecutive atoms (coalesced rows), a fixed butterfly at the end.
constexpr int kGradWarps = 8;
__global__ void __launch_bounds__(32 * kGradWarps) k64_grad_partial(const F64Args a) {
    const int c = blockIdx.x, N = a.N, T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA, H = a.H,
              D = a.D;
    const ParamLayout& L = a.L;
    const GradFields gf = grad_fields(a);
    const int a0 = c * kChunk, a1 = min(N, a0 + kChunk);
    const int lane = threadIdx.x & 31;
    for (int p = threadIdx.x >> 5; p < L.P; p += kGradWarps) {
        int sp, fa1, fb1 = -1, fa2 = -1, fb2 = -1;   // fa1 = -2: aE of the atom's configuration
        if (p < L.off_cR) {
            sp = p / L.mlp_stride;
            const int r = p % L.mlp_stride;
            if (r < H * D) {
                fa1 = gf.al + r / D;
                fb1 = gf.q + r % D;
                fa2 = gf.be + r / D;
                fb2 = gf.dq + r % D;
            } else if (r < H * D + H) {
                fa1 = gf.al + (r - H * D);
            } else if (r < H * D + 2 * H) {
                fa1 = gf.ga + (r - H * D - H);
            } else {
                fa1 = -2;
            }
        } else if (p < L.off_cA) {
            const int x = p - L.off_cR;
            sp = x / (T * NR * KR);
            const int t2 = (x / (NR * KR)) % T, n = (x / KR) % NR, k = x % KR;
            fa1 = gf.rho + n;
            fb1 = gf.F + t2 * KR + k;
            fa2 = gf.p + n;
            fb2 = gf.DF + t2 * KR + k;
        } else {
            const int x = p - L.off_cA;
            sp = x / (T * NA * KA);
            fa1 = gf.bins + x % (T * NA * KA);
        }
        double acc = 0.0;
        for (int i = a0 + lane; i < a1; i += 32) {
            if (a.type[i] != sp) continue;
            double v = fa1 == -2 ? a.aE[a.cfg[i]] : a.st[(size_t)fa1 * N + i];
            if (fb1 >= 0) v *= a.st[(size_t)fb1 * N + i];
            if (fa2 >= 0) v += a.st[(size_t)fa2 * N + i] * a.st[(size_t)fb2 * N + i];
            acc += v;
        }
        acc = group_sum<32>(acc);
        if (lane == 0) a.gpart[(size_t)c * L.P + p] = acc;
    }
}

__global__ void k64_grad_final(const F64Args a, int nchunk) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.L.P) return;
    double acc = 0.0;
    for (int c = 0; c < nchunk; ++c) acc += a.gpart[(size_t)c * a.L.P + p];
    a.grad[p] = acc;
}

}  // namespace

// lanes per atom: enough threads to fill the GPU (N G >= 2^17, about 1,024 per
// SM), with G in {1, 8, 32}; a function of N alone
int fp64_lanes_per_atom(int N) {
    if (N >= (1 << 17)) return 1;
    if (N >= (1 << 14)) return 8;
    return 32;
}

int fp64_grad_fields(const F64Args& a) { return grad_fields(a).total; }

int fp64_grad_chunks(int N) { return (N + kChunk - 1) / kChunk; }

cudaError_t launch_promote(const float* src, double* dst, int n, cudaStream_t st) {
    if (n > 0) k_promote<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

namespace {
template <class A>
cudaError_t launch_efv_t(const A& a, int max_chunks, double* e_tot, double* virial, cudaStream_t st) {
    if (a.N > 0) {
        const int G = fp64_lanes_per_atom(a.N);
        const int grid = (int)(((long long)a.N * G + kF64Block - 1) / kF64Block);
        if (G == 1) {
            k64_atom<1, A><<<grid, kF64Block, 0, st>>>(a);
            k64_force<1, A><<<grid, kF64Block, 0, st>>>(a);
        } else if (G == 8) {
            k64_atom<8, A><<<grid, kF64Block, 0, st>>>(a);
            k64_force<8, A><<<grid, kF64Block, 0, st>>>(a);
        } else {
            k64_atom<32, A><<<grid, kF64Block, 0, st>>>(a);
            k64_force<32, A><<<grid, kF64Block, 0, st>>>(a);
        }
    }
    if (max_chunks > 0) k64_chunk_reduce<A><<<max_chunks, kF64Red, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_final_reduce(a.B, a.chunk_start, a.partial, e_tot, virial, st);
}
}  // namespace

cudaError_t launch_efv_fp64(const F64Args& a, int max_chunks, double* e_tot, double* virial,
                            cudaStream_t st) {
    return launch_efv_t(a, max_chunks, e_tot, virial, st);
}

cudaError_t launch_efv_generic(const F32Args& a, int max_chunks, double* e_tot, double* virial,
                               cudaStream_t st) {
    return launch_efv_t(a, max_chunks, e_tot, virial, st);
}

cudaError_t launch_loss_fp64(const F64Args& a, int max_chunks, const double* e_tot, const double* vir,
                             const double* e_lbl, const double* f_lbl, const double* v_lbl, const float* w,
                             int mode, double* lam, double* aE, double* mu, double* loss, cudaStream_t st) {
    // the per-chunk force sums reuse the evaluation's partials (consumed by then)
    if (max_chunks > 0) k64_loss_atoms<<<max_chunks, kF64Red, 0, st>>>(a, f_lbl, w[1], lam, a.partial);
    k64_loss_cfg<<<1, kF64Red, 0, st>>>(a, a.partial, e_tot, vir, e_lbl, v_lbl, w[0], w[1], w[2], mode, aE, mu,
                                        loss);
    return cudaGetLastError();
}

cudaError_t launch_grad_fp64(const F64Args& a, cudaStream_t st) {
    if (a.N > 0) {
        const int G = fp64_lanes_per_atom(a.N);
        const int grid = (int)(((long long)a.N * G + kF64Block - 1) / kF64Block);
        if (G == 1) k64_grad_atom<1><<<grid, kF64Block, 0, st>>>(a);
        else if (G == 8) k64_grad_atom<8><<<grid, kF64Block, 0, st>>>(a);
        else k64_grad_atom<32><<<grid, kF64Block, 0, st>>>(a);
        k64_grad_partial<<<fp64_grad_chunks(a.N), 32 * kGradWarps, 0, st>>>(a);
    }
    k64_grad_final<<<(a.L.P + 255) / 256, 256, 0, st>>>(a, fp64_grad_chunks(a.N));
    return cudaGetLastError();
}

}  // namespace nep
