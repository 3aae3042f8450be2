// FP64 evaluation of energies, forces and virial.
//
// The operators of Section 3.2 run in float64 as well as float32.  This path
// computes Eqs. 1-4 and 11-17 with every intermediate in double: positions
// (FP32 inputs) are promoted, the parameters are FP64, and pairs are kept by
// r < rc in double.  Hyper-parameters are runtime values.  G lanes per atom
// split its neighbour list: G = 1 once N fills the GPU, up to a warp for a
// few hundred atoms, so that small systems still reach every SM.  Two
// passes over the list:
//   k64_atom  : q_n (Eq. 11), S_nlm and q_nl (Eqs. 16-17), q4_n, the network
//               (Eq. 2), E_i, dE_i/dq_n (radial) and R_nlm = dE_i/dS_nlm
//   k64_force : F_i = sum_j [dE_i/dr_ij - dE_j/dr_ji] (Eq. 3), each pair
//               derivative recomputed from its owner's dE/dq and R; per-atom
//               virial W_i = -sum_j dE_i/dr_ij (x) r_ij (Eq. 4)
// then FP64 sums per 1,024-atom chunk and per configuration in a fixed order.
// Lane partials are combined by an xor butterfly, whose fixed tree leaves
// the same bits in every lane of the group; every pair term is evaluated by
// both of its atoms, so nothing is scattered, and for a given N (which fixes
// G) the result is deterministic.
#include <cuda_runtime.h>

#include "nep_device.cuh"
#include "nep_internal.h"

namespace nep {
namespace {

constexpr int kF64Block = 128;
constexpr int kF64MaxD = kF64MaxN * 6;   // n_rad + 5 n_ang
constexpr double kPi = 3.141592653589793;

// Q_k(r) and dQ_k/dr for k < K at r < rc: Q_k = (T_k(x) + 1)/2 f_c(r),
// x = 2(r/rc - 1)^2 - 1, f_c = (1 + cos(pi r/rc))/2 (Eqs. 12-15)
__device__ void basis64(double r, double rc, int K, double* f, double* fp) {
    const double z = r / rc;
    double sp, cp;
    sincospi(z, &sp, &cp);
    const double fc2 = 0.25 * (1.0 + cp);                 // f_c / 2
    const double dfc2 = -0.25 * kPi / rc * sp;            // (d f_c/dr) / 2
    const double t = z - 1.0, x = 2.0 * t * t - 1.0, dx = 4.0 * t / rc;
    double Tm = 1.0, Tk = x, dTm = 0.0, dTk = 1.0;
    f[0] = 2.0 * fc2;
    fp[0] = 2.0 * dfc2;
    if (K > 1) {
        f[1] = (x + 1.0) * fc2;
        fp[1] = dx * fc2 + (x + 1.0) * dfc2;
    }
    for (int k = 2; k < K; ++k) {
        const double Tn = 2.0 * x * Tk - Tm;
        const double dTn = 2.0 * Tk + 2.0 * x * dTk - dTm;
        f[k] = (Tn + 1.0) * fc2;
        fp[k] = dTn * dx * fc2 + (Tn + 1.0) * dfc2;
        Tm = Tk; Tk = Tn; dTm = dTk; dTk = dTn;
    }
}

// r_ij = (r_j - r_i) + s L in double, with the list's image or the minimum image
__device__ int pair64(const F64Args& a, int i, int s, double xi, double yi, double zi, const double* L,
                      double& dx, double& dy, double& dz) {
    const int N = a.N;
    const int j = a.nbr[(size_t)s * N + i];
    const double ux = (double)a.pos[j] - xi, uy = (double)a.pos[N + j] - yi, uz = (double)a.pos[2 * N + j] - zi;
    double sx, sy, sz;
    if (a.shift) {
        int ix, iy, iz;
        unpack_shift(a.shift[(size_t)s * N + i], ix, iy, iz);
        sx = ix; sy = iy; sz = iz;
    } else {
        sx = -rint(ux / L[0]);
        sy = -rint(uy / L[1]);
        sz = -rint(uz / L[2]);
    }
    dx = ux + sx * L[0];
    dy = uy + sy * L[1];
    dz = uz + sz * L[2];
    return j;
}

// sum over the G aligned lanes of an atom; every lane receives the same bits.
// The shuffles name only the group's lanes: a group whose atom index is past
// N leaves as a whole, while the other groups of its warp go on.
template <int G>
__device__ __forceinline__ double group_sum(double v) {
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
}

// G divides 32 and kF64Block, so no group straddles a warp
template <int G>
__global__ void __launch_bounds__(kF64Block) k64_atom(const F64Args a) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    if (i >= a.N) return;
    const int N = a.N, T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA, H = a.H, D = a.D;
    const int ti = a.type[i], b = a.cfg[i];
    const double L[3] = {a.box[3 * b], a.box[3 * b + 1], a.box[3 * b + 2]};
    const double xi = a.pos[i], yi = a.pos[N + i], zi = a.pos[2 * N + i];
    double q[kF64MaxD], S[kF64MaxN * kLM], f[kF64MaxK], fp[kF64MaxK];
    for (int d = 0; d < D; ++d) q[d] = 0.0;
    for (int x = 0; x < NA * kLM; ++x) S[x] = 0.0;
    // this lane's pairs: list slots lane, lane + G, ...
    const int nc = a.cnt[i];
    for (int s = lane; s < nc; s += G) {
        double dx, dy, dz;
        const int j = pair64(a, i, s, xi, yi, zi, L, dx, dy, dz);
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (!(r < a.rc_rad)) continue;
        const int tj = a.type[j];
        basis64(r, a.rc_rad, KR, f, fp);
        const double* cR = a.prm + a.L.off_cR + (size_t)(ti * T + tj) * NR * KR;
        for (int n = 0; n < NR; ++n) {
            double g = 0.0;
            for (int k = 0; k < KR; ++k) g += cR[n * KR + k] * f[k];
            q[n] += g;
        }
        if (!(r < a.rc_ang)) continue;
        basis64(r, a.rc_ang, KA, f, fp);
        const double* cA = a.prm + a.L.off_cA + (size_t)(ti * T + tj) * NA * KA;
        const double ir = 1.0 / r;
        const HarmTermsT<double> ht = harm_terms(dx * ir, dy * ir, dz * ir);
        double Y[kLM];
        for (int m = 0; m < kLM; ++m) {
            double gx, gy, gz;
            harm_m(m, ht, Y[m], gx, gy, gz);
        }
        for (int n = 0; n < NA; ++n) {
            double g = 0.0;
            for (int k = 0; k < KA; ++k) g += cA[n * KA + k] * f[k];
            for (int m = 0; m < kLM; ++m) S[n * kLM + m] += g * Y[m];
        }
    }
    for (int n = 0; n < NR; ++n) q[n] = group_sum<G>(q[n]);
    for (int x = 0; x < NA * kLM; ++x) S[x] = group_sum<G>(S[x]);
    // q_nl = sum_m C_lm S_nlm^2 and q4_n = tr(A_n^3) (every lane of the group)
    for (int n = 0; n < NA; ++n) {
        for (int m = 0; m < kLM; ++m) {
            const double v = S[n * kLM + m];
            q[NR + n * 4 + lm_l(m) - 1] += (double)clm(m) * v * v;
        }
        if (a.H4) q[NR + NA * 4 + n] = fourbody<double>(S + n * kLM + 3, nullptr);
    }
    // network: E_i = w1 . tanh(W0 q + b0) + b1, dE/dq = W0^T (w1 (1 - t^2));
    // lane takes hidden units h = lane, lane + G, ...
    const double* W0 = a.prm + (size_t)ti * a.L.mlp_stride;
    const double* b0 = W0 + (size_t)H * D;
    const double* w1 = b0 + H;
    double E = 0.0;
    double pq[kF64MaxD];
    for (int d = 0; d < D; ++d) pq[d] = 0.0;
    for (int h = lane; h < H; h += G) {
        const double* w = W0 + (size_t)h * D;
        double z = b0[h];
        for (int d = 0; d < D; ++d) z += w[d] * q[d];
        const double th = tanh(z);
        E += w1[h] * th;
        const double c = w1[h] * (1.0 - th * th);
        for (int d = 0; d < D; ++d) pq[d] += c * w[d];
    }
    E = group_sum<G>(E) + w1[H];
    for (int d = 0; d < D; ++d) pq[d] = group_sum<G>(pq[d]);
    if (lane == 0) a.e[i] = E;
    for (int n = lane; n < NR; n += G) a.p[(size_t)n * N + i] = pq[n];
    // R_nlm = dE/dq_nl 2 C_lm S_nlm (+ dE/dq4_n dq4_n/dS_n2m), entries split over lanes
    for (int x = lane; x < NA * kLM; x += G) {
        const int n = x / kLM, m = x % kLM;
        double v = 2.0 * (double)clm(m) * pq[NR + n * 4 + lm_l(m) - 1] * S[x];
        if (a.H4 && m >= 3 && m < 8) {
            double J[5];
            fourbody<double>(S + n * kLM + 3, J);
            v += pq[NR + NA * 4 + n] * J[m - 3];
        }
        a.R[(size_t)x * N + i] = v;
    }
}

// dE_o/dr_oj for owner o of species to, neighbour species tn, distance r and
// unit vector u = r_oj / r
__device__ void pair_deriv(const F64Args& a, int o, int to, int tn, double r, const double* u, double* fo) {
    const int N = a.N, T = a.T, NR = a.NR, NA = a.NA, KR = a.KR, KA = a.KA;
    double f[kF64MaxK], fp[kF64MaxK];
    basis64(r, a.rc_rad, KR, f, fp);
    const double* cR = a.prm + a.L.off_cR + (size_t)(to * T + tn) * NR * KR;
    double gr = 0.0;
    for (int n = 0; n < NR; ++n) {
        double dg = 0.0;
        for (int k = 0; k < KR; ++k) dg += cR[n * KR + k] * fp[k];
        gr += a.p[(size_t)n * N + o] * dg;
    }
    fo[0] = gr * u[0];
    fo[1] = gr * u[1];
    fo[2] = gr * u[2];
    if (!(r < a.rc_ang)) return;
    basis64(r, a.rc_ang, KA, f, fp);
    const double* cA = a.prm + a.L.off_cA + (size_t)(to * T + tn) * NA * KA;
    const HarmTermsT<double> ht = harm_terms(u[0], u[1], u[2]);
    double Y[kLM], G[kLM][3];
    for (int m = 0; m < kLM; ++m) harm_m(m, ht, Y[m], G[m][0], G[m][1], G[m][2]);
    const double ir = 1.0 / r;
    for (int n = 0; n < NA; ++n) {
        double g = 0.0, gp = 0.0;
        for (int k = 0; k < KA; ++k) {
            g += cA[n * KA + k] * f[k];
            gp += cA[n * KA + k] * fp[k];
        }
        // d S_nlm / d r_oj = g'_n Y_m u + g_n (grad P_m - l P_m u) / r
        double sY = 0.0, slY = 0.0, sg[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < kLM; ++m) {
            const double Rv = a.R[(size_t)(n * kLM + m) * N + o];
            sY += Rv * Y[m];
            slY += Rv * lm_l(m) * Y[m];
            sg[0] += Rv * G[m][0];
            sg[1] += Rv * G[m][1];
            sg[2] += Rv * G[m][2];
        }
        for (int c = 0; c < 3; ++c) fo[c] += gp * sY * u[c] + g * ir * (sg[c] - slY * u[c]);
    }
}

template <int G>
__global__ void __launch_bounds__(kF64Block) k64_force(const F64Args a) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int lane = threadIdx.x % G;
    if (i >= a.N) return;
    const int N = a.N;
    const int ti = a.type[i], b = a.cfg[i];
    const double L[3] = {a.box[3 * b], a.box[3 * b + 1], a.box[3 * b + 2]};
    const double xi = a.pos[i], yi = a.pos[N + i], zi = a.pos[2 * N + i];
    double F[3] = {0.0, 0.0, 0.0}, W[9];
    for (int c = 0; c < 9; ++c) W[c] = 0.0;
    const int nc = a.cnt[i];
    for (int s = lane; s < nc; s += G) {
        double d[3];
        const int j = pair64(a, i, s, xi, yi, zi, L, d[0], d[1], d[2]);
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(r < a.rc_rad)) continue;
        const int tj = a.type[j];
        const double u[3] = {d[0] / r, d[1] / r, d[2] / r};
        const double v[3] = {-u[0], -u[1], -u[2]};
        double fij[3], fji[3];
        pair_deriv(a, i, ti, tj, r, u, fij);
        pair_deriv(a, j, tj, ti, r, v, fji);
        for (int c = 0; c < 3; ++c) F[c] += fij[c] - fji[c];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) W[3 * x + y] -= fij[x] * d[y];
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
// then warp shuffles and the warp sums in order
constexpr int kF64Red = 256;
__global__ void __launch_bounds__(kF64Red) k64_chunk_reduce(const F64Args a) {
    const int k = blockIdx.x, B = a.B, N = a.N;
    if (k >= a.chunk_start[B]) return;
    const int b = segment_of(a.chunk_start, B, k);
    const int a0 = a.atom_off[b] + (k - a.chunk_start[b]) * kChunk;
    const int a1 = min(a.atom_off[b + 1], a0 + kChunk);
    double acc[10];
    for (int c = 0; c < 10; ++c) acc[c] = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += kF64Red) {
        acc[0] += a.e[i];
        for (int c = 0; c < 9; ++c) acc[1 + c] += a.w[(size_t)c * N + i];
    }
    __shared__ double red[10][kF64Red / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int c = 0; c < 10; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int q = 0; q < kF64Red / 32; ++q) v += red[threadIdx.x][q];
        a.partial[(size_t)k * 10 + threadIdx.x] = v;
    }
}

__global__ void k_promote(const float* src, double* dst, int n) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < n) dst[x] = (double)src[x];
}

}  // namespace

// lanes per atom: enough threads to fill the GPU (N G >= 2^17, about 1,024 per
// SM), with G in {1, 8, 32}; a function of N alone
int fp64_lanes_per_atom(int N) {
    if (N >= (1 << 17)) return 1;
    if (N >= (1 << 14)) return 8;
    return 32;
}

cudaError_t launch_promote(const float* src, double* dst, int n, cudaStream_t st) {
    if (n > 0) k_promote<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_efv_fp64(const F64Args& a, int max_chunks, double* e_tot, double* virial,
                            cudaStream_t st) {
    if (a.N > 0) {
        const int G = fp64_lanes_per_atom(a.N);
        const int grid = (int)(((long long)a.N * G + kF64Block - 1) / kF64Block);
        if (G == 1) {
            k64_atom<1><<<grid, kF64Block, 0, st>>>(a);
            k64_force<1><<<grid, kF64Block, 0, st>>>(a);
        } else if (G == 8) {
            k64_atom<8><<<grid, kF64Block, 0, st>>>(a);
            k64_force<8><<<grid, kF64Block, 0, st>>>(a);
        } else {
            k64_atom<32><<<grid, kF64Block, 0, st>>>(a);
            k64_force<32><<<grid, kF64Block, 0, st>>>(a);
        }
    }
    if (max_chunks > 0) k64_chunk_reduce<<<max_chunks, kF64Red, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_final_reduce(a.B, a.chunk_start, a.partial, e_tot, virial, st);
}

}  // namespace nep
