// Mixed-precision per-species network on the tensor cores (Section 2.3):
// E_i = sum_h w1[h] tanh(z_h) + b1, z = W0 q + b0, p = dE_i/dq = W0^T (w1 (1 - t^2)),
// with q and W0 in FP16 or BF16 and FP32 accumulation; tanh, the sum over h
// and everything after p stay FP32.
//
// All species are computed at once: W = [W0_0; W0_1; W0_2] (T*H x D), so
//   GEMM1  Z[16 x T*H] = Q[16 x D] W^T   (each atom keeps its species' block)
//   GEMM2  P[16 x D]   = G[16 x T*H] W   (G = w1 (1 - t^2) in the own block, 0 elsewhere)
// per warp and 16-atom tile, with mma.sync m16n8k16.  The FP32 accumulators of
// two adjacent GEMM1 n-tiles are exactly the A fragment of one GEMM2 k-step.
#pragma once
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
    int wall, wallT, b0, w1, b1, cR, pst; // byte offsets
    int total;
};

template <class C>
NEP_HD TcLayout tc_layout(int H) {
    using Dm = TcDims<C>;
    TcLayout L;
    L.NT = C::T * H;
    L.NTp = (L.NT + 15) / 16 * 16;
    L.wstride = Dm::Kp + 8;               // conflict-free 32-bit fragment loads
    L.tstride = L.NTp + 8;
    int o = 0;
    L.wall = o;  o += 2 * L.NTp * L.wstride;
    L.wallT = o; o += 2 * Dm::Dn * L.tstride;
    o = (o + 15) / 16 * 16;
    L.b0 = o;    o += 4 * L.NTp;
    L.w1 = o;    o += 4 * L.NTp;
    L.b1 = o;    o += 4 * C::T;
    L.cR = o;    o += 4 * C::T * C::T * C::NR * C::KR;
    o = (o + 15) / 16 * 16;
    L.pst = o;   o += 4 * 4 * 16 * (Dm::Dn + 1);   // 4 warps x 16 rows x (Dn + 1)
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

template <class C, typename TIN>
__global__ void __launch_bounds__(128) k_mlp_tc(const EvalArgs a) {
    using Dm = TcDims<C>;
    constexpr int D = C::D, Kp = Dm::Kp, Dn = Dm::Dn, NR = C::NR, KR = C::KR, T = C::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int H = a.H, N = a.N;
    const TcLayout L = tc_layout<C>(H);
    TIN* wall = reinterpret_cast<TIN*>(smraw + L.wall);
    TIN* wallT = reinterpret_cast<TIN*>(smraw + L.wallT);
    float* b0s = reinterpret_cast<float*>(smraw + L.b0);
    float* w1s = reinterpret_cast<float*>(smraw + L.w1);
    float* b1s = reinterpret_cast<float*>(smraw + L.b1);
    float* cRs = reinterpret_cast<float*>(smraw + L.cR);
    const ParamLayout PL = param_layout(T, NR, C::NA, KR, C::KA, C::H4, H);
    // stage the stacked weights: wall[n][k] = W0[t][h][d] (n = t H + h, k = d), and its transpose
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
    for (int x = threadIdx.x; x < T * T * NR * KR; x += blockDim.x) cRs[x] = a.params[PL.off_cR + x];
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, tq = lane & 3;
    float* pst = reinterpret_cast<float*>(smraw + L.pst) + warp * 16 * (Dn + 1);
    const unsigned* q16 = reinterpret_cast<const unsigned*>(a.q16);
    const int ntiles = (N + 15) / 16;
    for (int tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
        const int r0 = tile * 16 + g, r1 = r0 + 8;
        const bool v0 = r0 < N, v1 = r1 < N;
        const int sp0 = v0 ? f2i(a.pos4[r0].w) : -1;
        const int sp1 = v1 ? f2i(a.pos4[r1].w) : -1;
        unsigned af[Kp / 16][4];
#pragma unroll
        for (int ks = 0; ks < Kp / 16; ++ks) {
            const int c = ks * 8 + tq;   // 32-bit word index of column 2*tq in this k-step
            af[ks][0] = v0 ? q16[(size_t)r0 * (Kp / 2) + c] : 0u;
            af[ks][1] = v1 ? q16[(size_t)r1 * (Kp / 2) + c] : 0u;
            af[ks][2] = v0 ? q16[(size_t)r0 * (Kp / 2) + c + 4] : 0u;
            af[ks][3] = v1 ? q16[(size_t)r1 * (Kp / 2) + c + 4] : 0u;
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
                // epilogue: own-species columns get tanh, the energy and w1 (1 - t^2)
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
        // energies: the four lanes of a quad hold partial sums of rows g and g + 8
        e0 += __shfl_xor_sync(0xffffffffu, e0, 1);
        e0 += __shfl_xor_sync(0xffffffffu, e0, 2);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 1);
        e1 += __shfl_xor_sync(0xffffffffu, e1, 2);
        if (tq == 0) {
            if (v0) a.e_atom[r0] = e0 + b1s[sp0];
            if (v1) a.e_atom[r1] = e1 + b1s[sp1];
        }
        // p rows through shared memory, then one lane per atom writes the
        // angular dE/dq and the species-projected radial adjoint
#pragma unroll
        for (int n2 = 0; n2 < Dn / 8; ++n2) {
            const int col = n2 * 8 + 2 * tq;
            pst[g * (Dn + 1) + col] = pacc[n2][0];
            pst[g * (Dn + 1) + col + 1] = pacc[n2][1];
            pst[(g + 8) * (Dn + 1) + col] = pacc[n2][2];
            pst[(g + 8) * (Dn + 1) + col + 1] = pacc[n2][3];
        }
        __syncwarp();
        if (lane < 16) {
            const int i = tile * 16 + lane;
            if (i < N) {
                const float* pr = pst + lane * (Dn + 1);
                const int ti = f2i(a.pos4[i].w);
                for (int d = NR; d < D; ++d) a.pang[(size_t)(d - NR) * N + i] = pr[d];
                for (int t = 0; t < T; ++t)
                    for (int k = 0; k < KR; ++k) {
                        float acc = 0.0f;
                        const float* c = cRs + ((ti * T + t) * NR) * KR + k;
                        for (int n = 0; n < NR; ++n) acc = fmaf(pr[n], c[n * KR], acc);
                        a.Pr[((size_t)i * T + t) * KR + k] = acc;
                    }
            }
        }
        __syncwarp();
    }
}

template <class C>
cudaError_t launch_mlp_tc_t(const EvalArgs& a, cudaStream_t st) {
    const int ntiles = (a.N + 15) / 16;
    if (ntiles == 0) return cudaSuccess;
    const TcLayout L = tc_layout<C>(a.H);
    int grid = (ntiles + 3) / 4;
    if (grid > 152 * 8) grid = 152 * 8;
    if (a.q16_kind == 2)
        k_mlp_tc<C, __nv_bfloat16><<<grid, 128, L.total, st>>>(a);
    else
        k_mlp_tc<C, __half><<<grid, 128, L.total, st>>>(a);
    return cudaGetLastError();
}

template <class C>
cudaError_t mlp_tc_init_t(int H) {
    const int smem = tc_layout<C>(H).total;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_mlp_tc<C, __half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
    return cudaFuncSetAttribute(k_mlp_tc<C, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}
#endif

}  // namespace nep
