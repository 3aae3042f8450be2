// Mixed-precision angular kernel: the per-species network (Section 2.3)
// E_i = sum_h w1[h] tanh(z_h) + b1, z = W0 q + b0, p = dE_i/dq = W0^T (w1 (1 - t^2))
// on the tensor cores with q and W0 in FP16 or BF16 and FP32 accumulation;
// descriptors, tanh, the sum over h, dE/dS and the forces stay FP32.
//
// All species are computed at once: W = [W0_0; W0_1; W0_2] (T*H x D), so
//   GEMM1  Z[16 x T*H] = Q[16 x D] W^T   (each atom keeps its species' block)
//   GEMM2  P[16 x D]   = G[16 x T*H] W   (G = w1 (1 - t^2) in the own block, 0 elsewhere)
// per warp and 16-atom tile, with mma.sync m16n8k16.  The FP32 accumulators of
// two adjacent GEMM1 n-tiles are exactly the A fragment of one GEMM2 k-step.
// Each thread computes its atom's descriptors, the warp runs the network for
// its 32 atoms out of shared memory, and each thread continues with its
// atom's angular pair forces.
#pragma once
#include <type_traits>

#include "nep_eval.cuh"

namespace nep {

template <class C>
struct TcDims {
    static constexpr int D = C::D;
    static constexpr int Kp = (D + 15) / 16 * 16;    // GEMM1 K
    static constexpr int Dn = (D + 7) / 8 * 8;       // GEMM2 N
};

struct TcLayout {
    int NT, NTp, wstride, tstride;        // columns T*H, padded to 16; smem row strides (halves)
    int coef, wall, wallT, b0, w1, b1, qst, pst, spc;   // byte offsets
    int total;
};

// shared memory: c coefficients (as in the FP32 image), stacked weights and
// their transpose, biases, and per-warp staging of q (16-bit), p and species
template <class C>
NEP_HD TcLayout tc_layout(int H) {
    using Dm = TcDims<C>;
    TcLayout L;
    L.NT = C::T * H;
    L.NTp = (L.NT + 15) / 16 * 16;
    L.wstride = Dm::Kp + 8;               // conflict-free 32-bit fragment loads
    L.tstride = L.NTp + 8;
    int o = 0;
    L.coef = o;  o += 4 * smem_layout<C>(H).W0;      // cA and cR blocks of the FP32 image
    o = (o + 15) / 16 * 16;
    L.wall = o;  o += 2 * L.NTp * L.wstride;
    L.wallT = o; o += 2 * Dm::Dn * L.tstride;
    o = (o + 15) / 16 * 16;
    L.b0 = o;    o += 4 * L.NTp;
    L.w1 = o;    o += 4 * L.NTp;
    L.b1 = o;    o += 4 * C::T;
    o = (o + 15) / 16 * 16;
    L.qst = o;   o += 2 * (kBlock / 32) * 32 * L.wstride;
    L.pst = o;   o += 4 * (kBlock / 32) * 32 * (Dm::Dn + 1);
    L.spc = o;   o += 4 * kBlock;
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

template <typename TIN>
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, unsigned b0, unsigned b1);
template <>
__device__ __forceinline__ void mma16816<__half>(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma16816<__nv_bfloat16>(float* d, const unsigned* a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <class C, typename TIN, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_angular_tc(const EvalArgs a) {
    using Dm = TcDims<C>;
    constexpr int D = C::D, Kp = Dm::Kp, Dn = Dm::Dn, NR = C::NR, NA = C::NA, KR = C::KR, T = C::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int H = a.H, N = a.N;
    const TcLayout L = tc_layout<C>(H);
    const SmemLayout sl = smem_layout<C>(H);
    float* sm = reinterpret_cast<float*>(smraw + L.coef);
    TIN* wall = reinterpret_cast<TIN*>(smraw + L.wall);
    TIN* wallT = reinterpret_cast<TIN*>(smraw + L.wallT);
    float* b0s = reinterpret_cast<float*>(smraw + L.b0);
    float* w1s = reinterpret_cast<float*>(smraw + L.w1);
    float* b1s = reinterpret_cast<float*>(smraw + L.b1);
    const ParamLayout PL = param_layout(T, NR, NA, KR, C::KA, C::H4, H);
    // c coefficients (cA, cR) into the padded image used by the FP32 helpers
    {
        const int nA = T * T * NA * C::KA;
        for (int x = threadIdx.x; x < nA; x += blockDim.x) {
            const int pair = x / (NA * C::KA), r = x % (NA * C::KA);
            sm[sl.cA + pair * C::SA + r] = a.params[PL.off_cA + x];
        }
        const int nR = T * T * NR * KR;
        for (int x = threadIdx.x; x < nR; x += blockDim.x) {
            const int pair = x / (NR * KR), r = x % (NR * KR);
            sm[sl.cR + pair * C::SR + r] = a.params[PL.off_cR + x];
        }
    }
    // stacked weights: wall[n][k] = W0[t][h][d] (n = t H + h, k = d), and its transpose
    for (int x = threadIdx.x; x < L.NTp * Kp; x += blockDim.x) {
        const int n = x / Kp, k = x % Kp;
        float v = 0.0f;
        if (n < L.NT && k < D) v = a.params[(n / H) * PL.mlp_stride + (n % H) * D + k];
        wall[n * L.wstride + k] = to_in<TIN>(v);
    }
    for (int x = threadIdx.x; x < Dn * L.NTp; x += blockDim.x) {
        const int n = x / L.NTp, k = x % L.NTp;
        float v = 0.0f;
        if (k < L.NT && n < D) v = a.params[(k / H) * PL.mlp_stride + (k % H) * D + n];
        wallT[n * L.tstride + k] = to_in<TIN>(v);
    }
    for (int x = threadIdx.x; x < L.NTp; x += blockDim.x) {
        float b = 0.0f, w = 0.0f;
        if (x < L.NT) {
            const int t = x / H, h = x % H;
            b = a.params[t * PL.mlp_stride + H * D + h];
            w = a.params[t * PL.mlp_stride + H * D + H + h];
        }
        b0s[x] = b;
        w1s[x] = w;
    }
    for (int t = threadIdx.x; t < T; t += blockDim.x) b1s[t] = a.params[t * PL.mlp_stride + H * D + 2 * H];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (N + kBlock - 1) / kBlock;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int i = tile * kBlock + threadIdx.x;
    const bool valid = i < N;
    TIN* qrow = reinterpret_cast<TIN*>(smraw + L.qst) + (warp * 32 + lane) * L.wstride;
    float* prow_base = reinterpret_cast<float*>(smraw + L.pst) + warp * 32 * (Dn + 1);
    int* spc = reinterpret_cast<int*>(smraw + L.spc) + warp * 32;

    // 1. descriptors of this thread's atom; S parked in memory, q staged 16-bit
    const int ti = valid ? f2i(a.pos4[i].w) : -1;
    {
        float q[D];
#pragma unroll
        for (int d = 0; d < D; ++d) q[d] = 0.0f;
        if (valid) {
            radial_q<C>(a, sm, sl, ti, i, q);
            float S[NA][kLM];
            angular_S<C>(a, sm, sl, ti, i, S);
            angular_q<C>(S, q);
#pragma unroll
            for (int n = 0; n < NA; ++n)
#pragma unroll
                for (int m = 0; m < kLM; ++m) a.S[(n * kLM + m) * N + i] = S[n][m];
        }
#pragma unroll
        for (int d = 0; d < Kp; d += 2) {
            const float x0 = d < D ? q[d] : 0.0f, x1 = d + 1 < D ? q[d + 1] : 0.0f;
            *reinterpret_cast<unsigned*>(qrow + d) = pack2<TIN>(x0, x1);
        }
        spc[lane] = ti;
    }
    __syncwarp();

    // 2. the warp's network on the tensor cores, two 16-atom tiles
    const int g = lane >> 2, tq = lane & 3;
    const int wbase = tile * kBlock + warp * 32;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        const int r0 = mt * 16 + g, r1 = r0 + 8;
        const int sp0 = spc[r0], sp1 = spc[r1];
        const unsigned* q0 = reinterpret_cast<const unsigned*>(
            reinterpret_cast<const TIN*>(smraw + L.qst) + (warp * 32 + r0) * L.wstride);
        const unsigned* q1 = reinterpret_cast<const unsigned*>(
            reinterpret_cast<const TIN*>(smraw + L.qst) + (warp * 32 + r1) * L.wstride);
        unsigned af[Kp / 16][4];
#pragma unroll
        for (int ks = 0; ks < Kp / 16; ++ks) {
            af[ks][0] = q0[ks * 8 + tq];
            af[ks][1] = q1[ks * 8 + tq];
            af[ks][2] = q0[ks * 8 + tq + 4];
            af[ks][3] = q1[ks * 8 + tq + 4];
        }
        float e0 = 0.0f, e1 = 0.0f;
        float pacc[Dn / 8][4];
#pragma unroll
        for (int n2 = 0; n2 < Dn / 8; ++n2)
#pragma unroll
            for (int c = 0; c < 4; ++c) pacc[n2][c] = 0.0f;
        for (int kk = 0; kk < L.NTp / 16; ++kk) {
            unsigned a2[4];
#pragma unroll
            for (int hf = 0; hf < 2; ++hf) {
                const int nt = 2 * kk + hf;
                float c4[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                const unsigned* wrow = reinterpret_cast<const unsigned*>(wall + (nt * 8 + g) * L.wstride);
#pragma unroll
                for (int ks = 0; ks < Kp / 16; ++ks)
                    mma16816<TIN>(c4, af[ks], wrow[ks * 8 + tq], wrow[ks * 8 + tq + 4]);
                float s4[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int col = nt * 8 + 2 * tq + (c & 1);
                    const int sp = col < L.NT ? col / H : -2;
                    const int spr = (c < 2) ? sp0 : sp1;
                    float s = 0.0f;
                    if (sp == spr) {
                        const float th = tanh_f(c4[c] + b0s[col]);
                        const float w = w1s[col];
                        if (c < 2) e0 = fmaf(w, th, e0); else e1 = fmaf(w, th, e1);
                        s = w * (1.0f - th * th);
                    }
                    s4[c] = s;
                }
                a2[2 * hf + 0] = pack2<TIN>(s4[0], s4[1]);
                a2[2 * hf + 1] = pack2<TIN>(s4[2], s4[3]);
            }
#pragma unroll
            for (int n2 = 0; n2 < Dn / 8; ++n2) {
                const unsigned* trow = reinterpret_cast<const unsigned*>(wallT + (n2 * 8 + g) * L.tstride);
                mma16816<TIN>(pacc[n2], a2, trow[kk * 8 + tq], trow[kk * 8 + tq + 4]);
            }
        }
        e0 += __shfl_xor_sync(0xffffffffu, e0, 1);
        e0 += __shfl_xor_sync(0xffffffffu, e0, 2);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
        if (tq == 0) {
            if (wbase + r0 < N) a.e_atom[wbase + r0] = e0 + b1s[sp0];
            if (wbase + r1 < N) a.e_atom[wbase + r1] = e1 + b1s[sp1];
        }
#pragma unroll
        for (int n2 = 0; n2 < Dn / 8; ++n2) {
            const int col = n2 * 8 + 2 * tq;
            prow_base[r0 * (Dn + 1) + col] = pacc[n2][0];
            prow_base[r0 * (Dn + 1) + col + 1] = pacc[n2][1];
            prow_base[r1 * (Dn + 1) + col] = pacc[n2][2];
            prow_base[r1 * (Dn + 1) + col + 1] = pacc[n2][3];
        }
    }
    __syncwarp();

    // 3. this thread's atom: projected radial adjoint, dE/dS, angular forces
    if (valid) {
    const float* p = prow_base + lane * (Dn + 1);
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
    float Sb[NA][kLM];
    make_Sb<C>(Sb, [&](int n, int m) { return a.S[(n * kLM + m) * N + i]; },
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
    __syncwarp();   // the staging rows are rewritten by the next tile
    }
}

template <class C, typename TIN>
void launch_angular_tc_v(const EvalArgs& a, cudaStream_t st, int v, int ntiles, size_t smem) {
    constexpr int K = sizeof(TIN) == 2 && std::is_same<TIN, __half>::value ? 1 : 2;
    if (v == 1)
        k_angular_tc<C, TIN, 3><<<persistent_grid(ntiles, resident_blocks<C, 3, K>()), kBlock, smem, st>>>(a);
    else if (v == 2)
        k_angular_tc<C, TIN, 4><<<persistent_grid(ntiles, resident_blocks<C, 4, K>()), kBlock, smem, st>>>(a);
    else
        k_angular_tc<C, TIN, 2><<<persistent_grid(ntiles, resident_blocks<C, 2, K>()), kBlock, smem, st>>>(a);
}

template <class C>
cudaError_t launch_angular_tc_t(const EvalArgs& a, cudaStream_t st, int v) {
    const int ntiles = (a.N + kBlock - 1) / kBlock;
    if (ntiles == 0) return cudaSuccess;
    const size_t smem = tc_layout<C>(a.H).total;
    if (a.q16_kind == 2)
        launch_angular_tc_v<C, __nv_bfloat16>(a, st, v, ntiles, smem);
    else
        launch_angular_tc_v<C, __half>(a, st, v, ntiles, smem);
    return cudaGetLastError();
}

template <class C, typename TIN, int MINB>
cudaError_t tc_init_one(int smem) {
    constexpr int K = std::is_same<TIN, __half>::value ? 1 : 2;
    cudaError_t e = cudaFuncSetAttribute(k_angular_tc<C, TIN, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident_blocks<C, MINB, K>(), k_angular_tc<C, TIN, MINB>,
                                                         kBlock, smem);
}
template <class C, typename TIN>
cudaError_t tc_init_v(int smem) {
    cudaError_t e;
    if ((e = tc_init_one<C, TIN, 2>(smem))) return e;
    if ((e = tc_init_one<C, TIN, 3>(smem))) return e;
    return tc_init_one<C, TIN, 4>(smem);
}

// the angular kernel of the model's precision
template <class C>
cudaError_t launch_angular_any_t(const EvalArgs& a, cudaStream_t st, int v) {
    return a.q16_kind ? launch_angular_tc_t<C>(a, st, v) : launch_angular_t<C>(a, st, v);
}

template <class C>
cudaError_t mlp_tc_init_t(int H) {
    const int smem = tc_layout<C>(H).total;
    cudaError_t e;
    if ((e = tc_init_v<C, __half>(smem))) return e;
    return tc_init_v<C, __nv_bfloat16>(smem);
}
#endif

}  // namespace nep
