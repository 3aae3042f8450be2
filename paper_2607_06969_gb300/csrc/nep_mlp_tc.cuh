// Mixed-precision angular kernel: the per-species network (Section 2.3)
//   E_i = sum_h w1[h] tanh(z_h) + b1,  z = W0 q + b0,  p = dE_i/dq = W0^T (w1 (1 - t^2))
// on the 5th-generation tensor cores (tcgen05.mma, kind::f16) with q and W0
// in FP16 or BF16 and FP32 accumulation in tensor memory; descriptors, tanh,
// the sum over h, dE/dS and the forces stay FP32.
//
// One CTA owns a tile of 128 atoms (persistent over tiles):
//   1. each thread computes its atom's q and S_nlm (FP32); S is parked in the
//      thread's TMEM lane (or in global memory for the smaller register
//      budgets, whose CTAs cannot all hold it in TMEM);
//   2. the 128 q rows are written to shared memory in species order, one
//      16-bit row each, as the A operand (M = 128, K = D padded to 16);
//   3. GEMM1, one MMA over the stacked species Z[128 x T Hp] = Q W^T when its
//      accumulator fits beside S in tensor memory, else once per species s
//      present in the tile:
//        Z_s[128 x Hp] = Q[128 x Kp] W0_s^T      (accumulator in TMEM)
//      the threads whose row has species s read their row of Z_s (their own
//      TMEM lane), form tanh, the energy and g = w1 (1 - t^2) (registers);
//   4. the g rows are written in the block of their species of a stacked
//      A operand G[128 x T Hp] (zeros elsewhere), and GEMM2
//        P[128 x Dn] = G W^T,   W[d][s Hp + h] = W0_s[h][d]
//      gives every row's dE/dq;
//   5. each thread takes its atom's p from shared memory and continues with
//      the species-projected radial adjoint, dE/dS and the angular pair
//      forces, exactly as the FP32 kernel.
// Species order keeps most warps on one species, so each thread reads only
// its own species' H columns of Z.  Operands use the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix).
#pragma once
#include <type_traits>

#include "nep_eval.cuh"

namespace nep {

template <class C>
struct Tc5Dims {
    static constexpr int D = C::D;
    static constexpr int Kp = (D + 15) / 16 * 16;     // GEMM1 K, GEMM2 N
};

struct Tc5Layout {
    int Hp, NTp, accC, sCol, cols;                  // TMEM: accumulators at 0, S at sCol
    int single;                                     // GEMM1 for all species at once
    int coef, B1, B2, b0, w1, b1, U, wcnt, rowA, rowS, bar, slot;   // byte offsets
    int total;
};

// shared memory: c coefficients (as in the FP32 image), W0 per species as the
// GEMM1 B operand, the stacked transpose as the GEMM2 B operand, biases, one
// union buffer for Q / G / P, the species sort, the mbarrier and TMEM slot
template <class C>
NEP_HD Tc5Layout tc5_layout(int H, bool s_in_tmem) {
    constexpr int Kp = Tc5Dims<C>::Kp;
    Tc5Layout L;
    L.Hp = (H + 15) / 16 * 16;
    L.NTp = C::T * L.Hp;
    // one GEMM1 over the stacked species when its NTp accumulator columns fit
    // beside S in the 256 columns a CTA may hold (two CTAs per SM), else one
    // GEMM1 of Hp columns per species
    const int sCols = s_in_tmem ? C::NA * kLM : 0;
    const int accAll = L.NTp > Kp ? L.NTp : Kp;
    L.single = (L.NTp <= 256 && accAll + sCols <= 256) ? 1 : 0;
    L.accC = L.single ? accAll : (L.Hp > Kp ? L.Hp : Kp);
    L.sCol = L.accC;
    L.cols = (int)tc5::tmem_cols(L.accC + sCols);
    auto al = [](int x) { return (x + 127) / 128 * 128; };
    int o = 0;
    L.coef = o; o = al(o + 4 * smem_layout<C>(H).W0);     // cA and cR blocks of the FP32 image
    L.B1 = o;   o = al(o + 2 * L.NTp * Kp);
    L.B2 = o;   o = al(o + 2 * Kp * L.NTp);
    L.b0 = o;   o = al(o + 4 * L.NTp);
    L.w1 = o;   o = al(o + 4 * L.NTp);
    L.b1 = o;   o = al(o + 4 * C::T);
    const int uq = 2 * kBlock * Kp, ug = 2 * kBlock * L.NTp, up = 4 * kBlock * (Kp + 1);
    L.U = o;    o = al(o + (uq > ug ? (uq > up ? uq : up) : (ug > up ? ug : up)));
    L.wcnt = o; o = al(o + 4 * (kBlock / 32) * (C::T + 1));
    L.rowA = o; o = al(o + 4 * kBlock);
    L.rowS = o; o = al(o + 4 * kBlock);
    L.bar = o;  o = al(o + 8);
    L.slot = o; o = al(o + 4);
    L.total = o;
    return L;
}

#if defined(__CUDACC__)
template <typename TIN>
__device__ __forceinline__ unsigned pack2(float x, float y);
template <>
__device__ __forceinline__ unsigned pack2<__half>(float x, float y) {
    __half2 v = __floats2half2_rn(x, y);
    return *reinterpret_cast<unsigned*>(&v);
}
template <>
__device__ __forceinline__ unsigned pack2<__nv_bfloat16>(float x, float y) {
    __nv_bfloat162 v = __floats2bfloat162_rn(x, y);
    return *reinterpret_cast<unsigned*>(&v);
}
template <typename TIN>
__device__ __forceinline__ TIN to_in(float x);
template <>
__device__ __forceinline__ __half to_in<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_in<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// tanh on the SFU (tanh.approx.f32, relative error about 2^-11): the
// mixed-precision network's operands are 16-bit, whose rounding (2^-11 for
// FP16, 2^-8 for BF16) already sets the scale of its error
__device__ __forceinline__ float tanh_sfu(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// polls of an mbarrier before the kernel gives up (flags status[3] bit 1)
constexpr int kMbarPolls = 1 << 20;
// largest hidden width of the mixed-precision network (g of one row in registers)
constexpr int kTcMaxH = kTcMaxHidden;

// S_nlm lives in TMEM for the 255-register variant only
template <int MINB>
NEP_HD constexpr bool tc5_s_in_tmem() { return MINB == 2; }

template <class C, typename TIN, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_angular_tc(const EvalArgs a) {
    constexpr int D = C::D, Kp = Tc5Dims<C>::Kp, NR = C::NR, NA = C::NA, KR = C::KR, T = C::T;
    constexpr bool STM = tc5_s_in_tmem<MINB>();
    constexpr bool BF = std::is_same<TIN, __nv_bfloat16>::value;
    extern __shared__ __align__(128) unsigned char smraw[];
    const int H = a.H, N = a.N;
    const Tc5Layout L = tc5_layout<C>(H, STM);
    const int Hp = L.Hp, NTp = L.NTp;
    const SmemLayout sl = smem_layout<C>(H);
    float* sm = reinterpret_cast<float*>(smraw + L.coef);
    TIN* B1 = reinterpret_cast<TIN*>(smraw + L.B1);
    TIN* B2 = reinterpret_cast<TIN*>(smraw + L.B2);
    float* b0s = reinterpret_cast<float*>(smraw + L.b0);
    float* w1s = reinterpret_cast<float*>(smraw + L.w1);
    float* b1s = reinterpret_cast<float*>(smraw + L.b1);
    unsigned char* U = smraw + L.U;
    int* wcnt = reinterpret_cast<int*>(smraw + L.wcnt);
    int* rowA = reinterpret_cast<int*>(smraw + L.rowA);
    int* rowS = reinterpret_cast<int*>(smraw + L.rowS);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smraw + L.bar);
    uint32_t* slot = reinterpret_cast<uint32_t*>(smraw + L.slot);
    const ParamLayout PL = param_layout(T, NR, NA, KR, C::KA, C::H4, H);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- model image (once per CTA) ----
    {
        const int nA = T * T * NA * C::KA;
        for (int x = tid; x < nA; x += kBlock) {
            const int pair = x / (NA * C::KA), r = x % (NA * C::KA);
            sm[sl.cA + pair * C::SA + r] = a.params[PL.off_cA + x];
            sm[sl.cA2 + pair * C::SA + pair_index<C::KA>(r / C::KA, r % C::KA)] = a.params[PL.off_cA + x];
        }
        const int nR = T * T * NR * KR;
        for (int x = tid; x < nR; x += kBlock) {
            const int pair = x / (NR * KR), r = x % (NR * KR);
            sm[sl.cR + pair * C::SR + r] = a.params[PL.off_cR + x];
        }
    }
    // B1: row n = s Hp + h holds W0_s[h][0..D) (K = Kp); B2: row d holds W0_s[h][d] at column s Hp + h
    for (int x = tid; x < NTp * Kp; x += kBlock) {
        const int n = x / Kp, k = x % Kp, s = n / Hp, h = n % Hp;
        const float v = (h < H && k < D) ? a.params[s * PL.mlp_stride + h * D + k] : 0.0f;
        B1[tc5::cm_offset(n, k, Kp)] = to_in<TIN>(v);
    }
    for (int x = tid; x < Kp * NTp; x += kBlock) {
        const int d = x / NTp, n = x % NTp, s = n / Hp, h = n % Hp;
        const float v = (h < H && d < D) ? a.params[s * PL.mlp_stride + h * D + d] : 0.0f;
        B2[tc5::cm_offset(d, n, NTp)] = to_in<TIN>(v);
    }
    for (int x = tid; x < NTp; x += kBlock) {
        const int s = x / Hp, h = x % Hp;
        b0s[x] = h < H ? a.params[s * PL.mlp_stride + H * D + h] : 0.0f;
        w1s[x] = h < H ? a.params[s * PL.mlp_stride + H * D + H + h] : 0.0f;
    }
    for (int t = tid; t < T; t += kBlock) b1s[t] = a.params[t * PL.mlp_stride + H * D + 2 * H];
    if (warp == 0) tc5::alloc(slot, (uint32_t)L.cols);
    if (tid == 0) tc5::mbar_init(bar, 1);
    tc5::fence_async_smem();
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    const uint32_t tbase = *slot;
    const uint32_t tlane = tc5::lane_addr(tbase, warp, 0);       // this thread's lane, column 0
    const uint32_t uA = tc5::smem_addr(U), uB1 = tc5::smem_addr(B1), uB2 = tc5::smem_addr(B2);
    const bool single = L.single != 0;
    const uint32_t id1 = tc5::idesc_f16(128, single ? NTp : Hp, BF), id2 = tc5::idesc_f16(128, Kp, BF);
    uint32_t phase = 0;
    bool ok = true;

    const int ntiles = (N + kBlock - 1) / kBlock;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const int i = tile * kBlock + tid;
        const bool valid = i < N;
        const int ti = valid ? f2i(a.pos4[i].w) : 0;
        const int key = valid ? ti : T;              // invalid atoms sort last

        // 1. descriptors; S to the TMEM lane or to global memory
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
            if constexpr (STM) {
                __syncwarp();
                const float* Sf = &S[0][0];
#pragma unroll
                for (int c = 0; c < NA * kLM; c += 8) tc5::st8(tlane + L.sCol + c, Sf + c);
            } else if (valid) {
#pragma unroll
                for (int n = 0; n < NA; ++n)
#pragma unroll
                    for (int m = 0; m < kLM; ++m) a.S[(n * kLM + m) * N + i] = S[n][m];
            }
        }

        // 2. species order: row = rank of (key, tid)
        __syncthreads();                 // the previous tile's reads of U and wcnt are done
        unsigned mine = 0;
#pragma unroll
        for (int s = 0; s <= T; ++s) {
            const unsigned b = __ballot_sync(0xffffffffu, key == s);
            if (key == s) mine = b;
            if (lane == 0) wcnt[warp * (T + 1) + s] = __popc(b);
        }
        __syncthreads();
        int tot[T + 1];
        int row = 0;
#pragma unroll
        for (int s = 0; s <= T; ++s) {
            int sum = 0;
            for (int w = 0; w < kBlock / 32; ++w) {
                const int c = wcnt[w * (T + 1) + s];
                sum += c;
                if (s == key && w < warp) row += c;
                if (s < key) row += c;
            }
            tot[s] = sum;
        }
        row += __popc(mine & ((1u << lane) - 1u));
        rowA[row] = tid;
        rowS[row] = key;
        {
            TIN* Q = reinterpret_cast<TIN*>(U);
#pragma unroll
            for (int k8 = 0; k8 < Kp; k8 += 8) {
                uint4 v;
                v.x = pack2<TIN>(k8 + 0 < D ? q[k8 + 0] : 0.0f, k8 + 1 < D ? q[k8 + 1] : 0.0f);
                v.y = pack2<TIN>(k8 + 2 < D ? q[k8 + 2] : 0.0f, k8 + 3 < D ? q[k8 + 3] : 0.0f);
                v.z = pack2<TIN>(k8 + 4 < D ? q[k8 + 4] : 0.0f, k8 + 5 < D ? q[k8 + 5] : 0.0f);
                v.w = pack2<TIN>(k8 + 6 < D ? q[k8 + 6] : 0.0f, k8 + 7 < D ? q[k8 + 7] : 0.0f);
                *reinterpret_cast<uint4*>(Q + tc5::cm_offset(row, k8, Kp)) = v;
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();

        // 3. GEMM1 per species; this thread now serves sorted row `tid`
        const int rs = rowS[tid];
        float E = 0.0f;
        unsigned g2[kTcMaxH / 2];      // packed g of the own species (Hp <= kTcMaxH)
#pragma unroll
        for (int c = 0; c < kTcMaxH / 2; ++c) g2[c] = 0u;
        bool issued = false;
        for (int s = 0; s < T; ++s) {
            if (tot[s] == 0) continue;
            if (!single || !issued) {
                issued = true;
                // single: B = all T Hp rows of W0, once per tile; else species s's Hp rows
                if (tid == 0) {
                    const uint32_t b0 = single ? 0u : (uint32_t)(s * Hp * Kp * 2);
                    for (int ks = 0; ks < Kp / 16; ++ks)
                        tc5::mma_f16(tbase, tc5::smem_desc(uA + ks * 256, 128, Kp * 16),
                                     tc5::smem_desc(uB1 + b0 + ks * 256, 128, Kp * 16), id1, ks > 0);
                    tc5::commit(bar);
                }
                const bool got = tc5::mbar_wait(bar, phase, kMbarPolls);
                phase ^= 1u;
                if (!__syncthreads_and(got)) {
                    ok = false;
                    break;
                }
                tc5::fence_after();
            }
            const int zc = single ? s * Hp : 0;          // species s's first accumulator column
            if (__ballot_sync(0xffffffffu, rs == s) != 0u) {
                for (int c = 0; c < Hp; c += 16) {
                    float z[16];
                    __syncwarp();
                    tc5::ld16(tlane + zc + c, z);
                    tc5::wait_ld();
                    if (rs == s) {
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {   // b0 and w1 are zero for h >= H
                            const int h = c + j;
                            const float t0 = tanh_sfu(z[j] + b0s[s * Hp + h]);
                            const float t1 = tanh_sfu(z[j + 1] + b0s[s * Hp + h + 1]);
                            const float w0 = w1s[s * Hp + h], w1v = w1s[s * Hp + h + 1];
                            E = fmaf(w0, t0, E);
                            E = fmaf(w1v, t1, E);
                            g2[(c + j) / 2] = pack2<TIN>(w0 * (1.0f - t0 * t0), w1v * (1.0f - t1 * t1));
                        }
                    }
                }
            }
            if (!single) {
                tc5::fence_before();
                __syncthreads();         // every read of this species' Z is done before the next GEMM1
                tc5::fence_after();
            }
        }
        if (!ok) break;
        if (single) {
            tc5::fence_before();
            __syncthreads();             // every read of Z is done before GEMM2 reuses the columns
            tc5::fence_after();
        }
        if (rs < T) a.e_atom[tile * kBlock + rowA[tid]] = E + b1s[rs];

        // 4. stacked G rows (Q is no longer read), then GEMM2
        {
            TIN* G = reinterpret_cast<TIN*>(U);
            for (int n8 = 0; n8 < NTp; n8 += 8) {
                const int s = n8 / Hp, h8 = n8 % Hp;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (s == rs) {
#pragma unroll
                    for (int c = 0; c < kTcMaxH / 2; c += 4) {
                        if (c * 2 == h8) v = make_uint4(g2[c], g2[c + 1], g2[c + 2], g2[c + 3]);
                    }
                }
                *reinterpret_cast<uint4*>(G + tc5::cm_offset(tid, n8, NTp)) = v;
            }
        }
        tc5::fence_async_smem();
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();
        if (tid == 0) {
            for (int ks = 0; ks < NTp / 16; ++ks)
                tc5::mma_f16(tbase, tc5::smem_desc(uA + ks * 256, 128, NTp * 16),
                             tc5::smem_desc(uB2 + ks * 256, 128, NTp * 16), id2, ks > 0);
            tc5::commit(bar);
        }
        {
            const bool got = tc5::mbar_wait(bar, phase, kMbarPolls);
            phase ^= 1u;
            if (!__syncthreads_and(got)) {   // G (aliased by P below) is no longer read once this passes
                ok = false;
                break;
            }
        }
        tc5::fence_after();
        float* P = reinterpret_cast<float*>(U);
        {
            const int dst = rowA[tid];
            for (int c = 0; c < Kp; c += 16) {
                float v[16];
                __syncwarp();
                tc5::ld16(tlane + c, v);
                tc5::wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) P[dst * (Kp + 1) + c + j] = v[j];
            }
        }
        tc5::fence_before();
        __syncthreads();
        tc5::fence_after();

        // 5. this thread's atom: projected radial adjoint, dE/dS, angular forces
        const float* p = P + tid * (Kp + 1);
        float Sb[NA][kLM];
        if constexpr (STM) {
            __syncwarp();
            float* Sf = &Sb[0][0];
#pragma unroll
            for (int c = 0; c < NA * kLM; c += 8) tc5::ld8(tlane + L.sCol + c, Sf + c);
            tc5::wait_ld();
        } else if (valid) {
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int m = 0; m < kLM; ++m) Sb[n][m] = a.S[(n * kLM + m) * N + i];
        }
        if (valid) {
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
#pragma unroll
                for (int k = 0; k < KR; ++k) a.Pr[(i * T + t) * KR + k] = acc[k];
            }
            make_Sb<C>(Sb, [&](int n, int m) { return Sb[n][m]; },
                       [&](int n, int l) { return p[NR + (l < 4 ? n * 4 + l : NA * 4 + n)]; });
            float Fx = 0.0f, Fy = 0.0f, Fz = 0.0f;
            float W[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) W[k] = 0.0f;
            angular_force<C, true>(a, sm, sl, ti, i, Sb, Fx, Fy, Fz, W);
            a.fpart[i] = Fx;
            a.fpart[N + i] = Fy;
            a.fpart[2 * N + i] = Fz;
#pragma unroll
            for (int k = 0; k < 9; ++k) a.wat[k * N + i] = W[k];
        }
    }
    if (!ok) {
        // a tensor-core completion never arrived: flag it, give the MMA in
        // flight one more bounded wait, then free the columns and return
        if (tid == 0 && a.status) atomicOr(a.status + 3, 2);
        tc5::mbar_wait(bar, phase ^ 1u, kMbarPolls);
    }
    tc5::fence_before();
    __syncthreads();
    tc5::fence_after();
    if (warp == 0) tc5::dealloc(tbase, (uint32_t)L.cols);
}

template <class C, typename TIN, int MINB>
void launch_angular_tc_v(const EvalArgs& a, cudaStream_t st, int ntiles) {
    constexpr int K = std::is_same<TIN, __half>::value ? 1 : 2;
    const size_t smem = tc5_layout<C>(a.H, tc5_s_in_tmem<MINB>()).total;
    k_angular_tc<C, TIN, MINB><<<persistent_grid(ntiles, resident_blocks<C, MINB, K>()), kBlock, smem, st>>>(a);
}

template <class C, typename TIN>
void launch_angular_tc_p(const EvalArgs& a, cudaStream_t st, int v, int ntiles) {
    if (v == 1)
        launch_angular_tc_v<C, TIN, 3>(a, st, ntiles);
    else if (v == 2)
        launch_angular_tc_v<C, TIN, 4>(a, st, ntiles);
    else
        launch_angular_tc_v<C, TIN, 2>(a, st, ntiles);
}

template <class C>
cudaError_t launch_angular_tc_t(const EvalArgs& a, cudaStream_t st, int v) {
    const int ntiles = (a.N + kBlock - 1) / kBlock;
    if (ntiles == 0) return cudaSuccess;
    if (a.q16_kind == 2)
        launch_angular_tc_p<C, __nv_bfloat16>(a, st, v, ntiles);
    else
        launch_angular_tc_p<C, __half>(a, st, v, ntiles);
    return cudaGetLastError();
}

template <class C, typename TIN, int MINB>
cudaError_t tc_init_one(int H) {
    constexpr int K = std::is_same<TIN, __half>::value ? 1 : 2;
    const Tc5Layout L = tc5_layout<C>(H, tc5_s_in_tmem<MINB>());
    cudaError_t e =
        cudaFuncSetAttribute(k_angular_tc<C, TIN, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e) return e;
    resident_blocks<C, MINB, K>() =
        resident_by_resources((const void*)k_angular_tc<C, TIN, MINB>, kBlock, L.total, L.cols);
    return cudaGetLastError();
}
template <class C, typename TIN>
cudaError_t tc_init_v(int H) {
    cudaError_t e;
    if ((e = tc_init_one<C, TIN, 2>(H))) return e;
    if ((e = tc_init_one<C, TIN, 3>(H))) return e;
    return tc_init_one<C, TIN, 4>(H);
}

// the angular kernel of the model's precision
template <class C>
cudaError_t launch_angular_any_t(const EvalArgs& a, cudaStream_t st, int v) {
    return a.q16_kind ? launch_angular_tc_t<C>(a, st, v) : launch_angular_t<C>(a, st, v);
}

template <class C>
cudaError_t mlp_tc_init_t(int H) {
    if (H > kTcMaxH) return cudaSuccess;     // such models run in FP32 only
    cudaError_t e;
    if ((e = tc_init_v<C, __half>(H))) return e;
    return tc_init_v<C, __nv_bfloat16>(H);
}
#endif

}  // namespace nep
