// Slab decomposition of one periodic configuration along x: the exchange
// step of a multi-GPU run of one large system.
//
// A rank owns the atoms with x in [lo, hi) and evaluates them together with
// the ghost atoms within `halo` of its slab, taking for each ghost the image
// that lies in [lo - halo, hi + halo).  With halo = 2 (rc + skin), every
// neighbour of an owned atom has its own complete neighbourhood in the local
// system, so the owned atoms' energies, forces and per-atom virials come out
// exactly as in the whole-system evaluation.
//   select  : owned atoms, then ghosts, each in atom order (counts per block
//             of 1,024 atoms, an exclusive scan of the block counts, then
//             ballot ranks within the block): deterministic
//   gather  : positions into the slab's local frame (x - (lo - halo) plus
//             the ghost's image), species alongside
//   scatter : the owned atoms' rows of a local [ncomp][n_local] array into a
//             whole-system [ncomp][N] array
#include <cuda_runtime.h>

#include "nep_internal.h"

namespace nep {
namespace {

constexpr int kDomBlock = 1024;

// 0: owned, 1: ghost (img = its image in units of Lx), -1: outside the window
__device__ __forceinline__ int dom_class(float x, float Lx, float lo, float hi, float halo, int& img) {
    img = 0;
    if (x >= lo && x < hi) return 0;
    for (int k = -1; k <= 1; ++k) {
        const float xs = x + (float)k * Lx;
        if ((xs >= lo - halo && xs < lo) || (xs >= hi && xs < hi + halo)) {
            img = k;
            return 1;
        }
    }
    return -1;
}

__global__ void __launch_bounds__(kDomBlock) k_dom_count(const float* __restrict__ pos, int N, float Lx, float lo,
                                                        float hi, float halo, int* bc) {
    const int i = blockIdx.x * kDomBlock + threadIdx.x;
    int img;
    const int c = i < N ? dom_class(pos[i], Lx, lo, hi, halo, img) : -1;
    const int own = __syncthreads_count(c == 0);
    const int gh = __syncthreads_count(c == 1);
    if (threadIdx.x == 0) {
        bc[2 * blockIdx.x] = own;
        bc[2 * blockIdx.x + 1] = gh;
    }
}

// exclusive scan of v over the 1,024 threads of the block; total = the sum
__device__ int block_exscan(int v, int* warp_sums, int& total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    total = warp_sums[31];
    return x - v + (w > 0 ? warp_sums[w - 1] : 0);
}

// one block: block offsets of the owned and the ghost atoms; counts[0] = owned,
// counts[1] = owned + ghosts
__global__ void __launch_bounds__(kDomBlock) k_dom_scan(const int* bc, int nb, int* boff, int* counts) {
    __shared__ int ws[32];
    int carry_o = 0, carry_g = 0;
    for (int base = 0; base < nb; base += kDomBlock) {
        const int b = base + threadIdx.x;
        const int vo = b < nb ? bc[2 * b] : 0, vg = b < nb ? bc[2 * b + 1] : 0;
        int to, tg;
        const int eo = block_exscan(vo, ws, to);
        const int eg = block_exscan(vg, ws, tg);
        if (b < nb) {
            boff[2 * b] = carry_o + eo;
            boff[2 * b + 1] = carry_g + eg;
        }
        carry_o += to;
        carry_g += tg;
    }
    if (threadIdx.x == 0) {
        counts[0] = carry_o;
        counts[1] = carry_o + carry_g;
    }
}

__global__ void __launch_bounds__(kDomBlock) k_dom_write(const float* __restrict__ pos, int N, float Lx, float lo,
                                                        float hi, float halo, const int* __restrict__ boff,
                                                        const int* __restrict__ counts, int* idx, int* img_out,
                                                        int cap) {
    __shared__ int wo[32], wg[32];
    const int i = blockIdx.x * kDomBlock + threadIdx.x;
    int img = 0;
    const int c = i < N ? dom_class(pos[i], Lx, lo, hi, halo, img) : -1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bo = __ballot_sync(0xffffffffu, c == 0), bg = __ballot_sync(0xffffffffu, c == 1);
    if (lane == 0) {
        wo[w] = __popc(bo);
        wg[w] = __popc(bg);
    }
    __syncthreads();
    if (c < 0) return;
    int before = 0;
    for (int q = 0; q < w; ++q) before += c == 0 ? wo[q] : wg[q];
    const int r = before + __popc((c == 0 ? bo : bg) & ((1u << lane) - 1u));
    const int at = c == 0 ? boff[2 * blockIdx.x] + r : counts[0] + boff[2 * blockIdx.x + 1] + r;
    if (at < cap) {
        idx[at] = i;
        if (img_out) img_out[at] = img;
    }
}

__global__ void k_dom_gather(const float* __restrict__ pos, const int* __restrict__ type, int N,
                             const int* __restrict__ idx, const int* __restrict__ img, int n_local, float Lx,
                             float x_origin, float* pl, int* tl) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_local) return;
    const int i = idx[l];
    pl[l] = (pos[i] + (float)img[l] * Lx) - x_origin;
    pl[n_local + l] = pos[N + i];
    pl[2 * n_local + l] = pos[2 * N + i];
    tl[l] = type[i];
}

__global__ void k_dom_scatter(const float* __restrict__ src, int n_local, int ncomp, const int* __restrict__ idx,
                              int n_owned, float* dst, int N) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n_owned) return;
    const int i = idx[l];
    for (int c = 0; c < ncomp; ++c) dst[(size_t)c * N + i] = src[(size_t)c * n_local + l];
}

// dst[c][l] = src[c][idx[l]], 32-bit words
__global__ void k_dom_take(const unsigned* __restrict__ src, int n_src, int ncomp, const int* __restrict__ idx,
                           int n, unsigned* __restrict__ dst) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int i = idx[l];
    for (int c = 0; c < ncomp; ++c) dst[(size_t)c * n + l] = src[(size_t)c * n_src + i];
}

// dst[c * stride + offset + l] = src[c][l]; component 0 (x) shifted by the
// whole box lengths that bring it nearest x_center, then taken relative to
// x_origin, when box_x > 0; every other word copied bit for bit
__global__ void k_dom_place(const unsigned* __restrict__ src, int n, int ncomp, float box_x, float x_center,
                            float x_origin, unsigned* __restrict__ dst, int stride, int offset) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    for (int c = 0; c < ncomp; ++c) {
        unsigned v = src[(size_t)c * n + l];
        if (c == 0 && box_x > 0.0f) {
            const float x = __uint_as_float(v);
            const float k = rintf(__fdiv_rn(__fsub_rn(x, x_center), box_x));
            v = __float_as_uint(__fsub_rn(__fsub_rn(x, __fmul_rn(k, box_x)), x_origin));
        }
        dst[(size_t)c * stride + offset + l] = v;
    }
}

inline int dom_blocks(int N) { return (N + kDomBlock - 1) / kDomBlock; }

}  // namespace

// block counts and block offsets, two ints each per block of 1,024 atoms
size_t domain_scratch_bytes(int N) { return 16 * (size_t)(dom_blocks(N) + 1); }

cudaError_t launch_domain_select(const float* pos, int N, float Lx, float lo, float hi, float halo, int* idx,
                                 int* img, int cap, int* counts, void* scratch, cudaStream_t st) {
    const int nb = dom_blocks(N);
    int* bc = static_cast<int*>(scratch);
    int* boff = bc + 2 * (nb + 1);
    if (nb > 0) k_dom_count<<<nb, kDomBlock, 0, st>>>(pos, N, Lx, lo, hi, halo, bc);
    k_dom_scan<<<1, kDomBlock, 0, st>>>(bc, nb, boff, counts);
    if (nb > 0) k_dom_write<<<nb, kDomBlock, 0, st>>>(pos, N, Lx, lo, hi, halo, boff, counts, idx, img, cap);
    return cudaGetLastError();
}

cudaError_t launch_domain_gather(const float* pos, const int* type, int N, const int* idx, const int* img,
                                 int n_local, float Lx, float x_origin, float* pos_local, int* type_local,
                                 cudaStream_t st) {
    if (n_local > 0)
        k_dom_gather<<<(n_local + 255) / 256, 256, 0, st>>>(pos, type, N, idx, img, n_local, Lx, x_origin,
                                                            pos_local, type_local);
    return cudaGetLastError();
}

cudaError_t launch_domain_take(const void* src, int n_src, int ncomp, const int* idx, int n, void* dst,
                               cudaStream_t st) {
    if (n > 0)
        k_dom_take<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const unsigned*>(src), n_src, ncomp, idx, n,
                                                    static_cast<unsigned*>(dst));
    return cudaGetLastError();
}

cudaError_t launch_domain_place(const void* src, int n, int ncomp, float box_x, float x_center, float x_origin,
                                void* dst, int stride, int offset, cudaStream_t st) {
    if (n > 0)
        k_dom_place<<<(n + 255) / 256, 256, 0, st>>>(static_cast<const unsigned*>(src), n, ncomp, box_x, x_center,
                                                     x_origin, static_cast<unsigned*>(dst), stride, offset);
    return cudaGetLastError();
}

cudaError_t launch_domain_scatter(const float* src, int n_local, int ncomp, const int* idx, int n_owned, float* dst,
                                  int N, cudaStream_t st) {
    if (n_owned > 0)
        k_dom_scatter<<<(n_owned + 255) / 256, 256, 0, st>>>(src, n_local, ncomp, idx, n_owned, dst, N);
    return cudaGetLastError();
}

}  // namespace nep
