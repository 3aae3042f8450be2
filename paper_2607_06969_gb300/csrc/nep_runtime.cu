// Model-independent kernels of libnep: input packing, the cell-list
// neighbour build, the deterministic force gather with FP64 reductions, and
// the velocity-Verlet updates.
#include <cuda_runtime.h>

#include "nep_device.cuh"
#include "nep_internal.h"

namespace nep {

namespace {

__device__ __forceinline__ void set_flag(int* status, int k) {
    if (status) atomicOr(status + k, 1);
}

// binary search: largest b with off[b] <= x, for off[0..B]
__device__ __forceinline__ int find_segment(const int* off, int B, int x) {
    int lo = 0, hi = B;   // invariant off[lo] <= x < off[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------------------ packing
__global__ void k_pack(const float* __restrict__ pos, const int* __restrict__ type,
                       const int* __restrict__ atom_off, int N, int B, int T, float4* pos4,
                       int* cfg, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int t = type[i];
    if (t < 0 || t >= T) {
        set_flag(status, 3);
        t = 0;
    }
    const float x = pos[i], y = pos[N + i], z = pos[2 * N + i];
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) set_flag(status, 3);
    pos4[i] = make_float4(x, y, z, __int_as_float(t));
    cfg[i] = find_segment(atom_off, B, i);
}

// exclusive scan of per-configuration chunk counts (one CTA)
__global__ void k_chunk_plan(const int* __restrict__ atom_off, int B, int* chunk_start) {
    __shared__ int carry;
    __shared__ int warp_sums[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < B; base += blockDim.x) {
        const int b = base + threadIdx.x;
        int v = 0;
        if (b < B) {
            const int n = atom_off[b + 1] - atom_off[b];
            v = (n + kChunk - 1) / kChunk;
        }
        // block inclusive scan
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += y;
            }
            warp_sums[lane] = s;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? warp_sums[w - 1] : 0);
        if (b < B) chunk_start[b] = carry + incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) chunk_start[B] = carry;
}

constexpr int kRedThreads = 256;

// (hi, lo) += x without rounding loss: Knuth's two-sum, in FP32.  The pair
// carries about 48 significant bits, so the per-thread and per-warp stages
// below are as exact as FP64 while running on the FP32 pipes (GB300 issues
// FP64 at a small fraction of the FP32 rate).
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// one CTA per reduction chunk (atoms of one configuration): sums of the
// energies and per-atom virials, each thread over a fixed atom subset in
// two-sum pairs, a fixed warp tree of pairs, then FP64 across the warps
__global__ void __launch_bounds__(kRedThreads) k_chunk_reduce(const EvalArgs a, FinishArgs f) {
    const int k = blockIdx.x;
    const int B = a.B, N = a.N;
    const int total = f.chunk_start[B];
    if (k >= total) return;
    const int b = find_segment(f.chunk_start, B, k);
    const int a0 = f.atom_off[b] + (k - f.chunk_start[b]) * kChunk;
    const int a1 = min(min(f.atom_off[b + 1], a0 + kChunk), f.n_owned);
    float hi[10], lo[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) hi[c] = lo[c] = 0.0f;
    for (int i = a0 + threadIdx.x; i < a1; i += kRedThreads) {
        two_sum_add(hi[0], lo[0], a.e_atom[i]);
#pragma unroll
        for (int c = 0; c < 9; ++c) two_sum_add(hi[1 + c], lo[1 + c], a.wat[(size_t)c * N + i]);
    }
    __shared__ double red[10][kRedThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
        float h = hi[c], l = lo[c];
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h, o);
            const float ol = __shfl_down_sync(0xffffffffu, l, o);
            two_sum_add(h, l, oh);
            l = __fadd_rn(l, ol);
        }
        if (lane == 0) red[c][w] = (double)h + (double)l;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) v += red[threadIdx.x][q];
        f.partial[(size_t)k * 10 + threadIdx.x] = v;
    }
}

// one block per configuration: threads take chunk partials k = t, t+256, ...
// and a fixed tree (warp shuffles, then the 8 warp sums in order) combines
// them, so the sum order never changes
__global__ void __launch_bounds__(kRedThreads) k_final_reduce(int B, const int* __restrict__ chunk_start,
                                                              const double* __restrict__ partial,
                                                              double* e_tot, double* virial) {
    const int b = blockIdx.x;
    if (b >= B) return;
    double acc[10];
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] = 0.0;
    for (int k = chunk_start[b] + threadIdx.x; k < chunk_start[b + 1]; k += kRedThreads)
#pragma unroll
        for (int c = 0; c < 10; ++c) acc[c] += partial[(size_t)k * 10 + c];
    __shared__ double red[10][kRedThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 10; ++c) {
        double v = acc[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[c][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        double v = 0.0;
        for (int q = 0; q < kRedThreads / 32; ++q) v += red[threadIdx.x][q];
        if (threadIdx.x == 0) {
            if (e_tot) e_tot[b] = v;
        } else if (virial) {
            virial[(size_t)b * 9 + threadIdx.x - 1] = v;
        }
    }
}

// ------------------------------------------------------- neighbour build
// Cells per edge: floor(L / ((rc + 1e-3) / kCellDiv)) (at least 1), reduced
// while the cell count of a configuration exceeds 2 N_b + 27.  The stencil
// half-width is the number of cells needed to reach rc + 1e-3 (kCellDiv for
// large boxes).  Cells of a third of the cutoff offer (7/3)^3 = 12.7
// cutoff-sized cells' worth of candidates before the per-row cut below
// (half the cutoff: 15.6; the whole cutoff: 27); measured at 900k atoms, the
// rebuild takes 1.31 ms with thirds and 1.54 ms with halves.  An atom in cell
// c sees cells c + d, d in [-half, half], with image shift floor((c + d) /
// nc): every (j, image) within the cutoff is visited exactly once.
constexpr float kCellMargin = 1e-3f;
// margin (A) on the list cutoff when cells beyond it are skipped
#ifndef NEP_PRUNE_MARGIN
#define NEP_PRUNE_MARGIN 0.01f
#endif
constexpr float kPruneMargin = NEP_PRUNE_MARGIN;
constexpr int kCellDiv = 3;
// per-atom row starts of the angular prefix, for the reverse-slot search:
// stencils of up to kMaxRows (x, y) rows, angular capacity below 256; one
// atom's starts take kRowStride bytes of the workspace
constexpr int kMaxRows = (2 * kCellDiv + 1) * (2 * kCellDiv + 1);
static_assert(kMaxRows < kRowStride, "row starts must fit one atom's stride");

__global__ void k_cell_plan(const float* __restrict__ box, const int* __restrict__ atom_off, int B,
                            float rc, CellPlan* plan, int* status) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int nb = atom_off[b + 1] - atom_off[b];
    float L[3] = {box[3 * b], box[3 * b + 1], box[3 * b + 2]};
    int nc[3];
    for (int d = 0; d < 3; ++d) {
        if (!(L[d] > 0.0f) || !isfinite(L[d])) {
            set_flag(status, 3);
            L[d] = 1.0f;
        }
        const float r = floorf(L[d] / ((rc + kCellMargin) / (float)kCellDiv));
        nc[d] = r < 1.0f ? 1 : (r > 1024.0f ? 1024 : (int)r);
    }
    const long long cap = 2LL * nb + 27;
    while ((long long)nc[0] * nc[1] * nc[2] > cap) {
        int m = 0;
        if (nc[1] > nc[m]) m = 1;
        if (nc[2] > nc[m]) m = 2;
        nc[m] -= 1;
    }
    CellPlan p;
    for (int d = 0; d < 3; ++d) {
        p.nc[d] = nc[d];
        const float cs = L[d] / (float)nc[d];
        p.half[d] = (int)ceilf((rc + kCellMargin) / cs);
        if (p.half[d] < 1) p.half[d] = 1;
    }
    p.base = nc[0] * nc[1] * nc[2];   // count here, prefix in k_plan_scan
    p.pad = 0;
    plan[b] = p;
}

__global__ void k_plan_scan(CellPlan* plan, int B) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int acc = 0;
    for (int b = 0; b < B; ++b) {
        const int c = plan[b].base;
        plan[b].base = acc;
        acc += c;
    }
}

__device__ __forceinline__ void cell_coords(const CellPlan& p, float x, float y, float z,
                                            const float* L, int* c) {
    const float v[3] = {x, y, z};
    for (int d = 0; d < 3; ++d) {
        int ci = (int)(v[d] * ((float)p.nc[d] / L[d]));
        ci = ci < 0 ? 0 : (ci >= p.nc[d] ? p.nc[d] - 1 : ci);
        c[d] = ci;
    }
}

__global__ void k_bin(const float* __restrict__ pos, const int* __restrict__ cfg,
                      const float* __restrict__ box, const CellPlan* __restrict__ plan, int N,
                      int* cell_of, int* rank, int* cell_cnt, int* status) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = cfg[i];
    const CellPlan p = plan[b];
    const float L[3] = {box[3 * b], box[3 * b + 1], box[3 * b + 2]};
    const float x = pos[i], y = pos[N + i], z = pos[2 * N + i];
    if (!(x >= 0.0f && x < L[0] && y >= 0.0f && y < L[1] && z >= 0.0f && z < L[2]))
        set_flag(status, 3);
    int c[3];
    cell_coords(p, x, y, z, L, c);
    const int id = p.base + (c[0] * p.nc[1] + c[1]) * p.nc[2] + c[2];
    cell_of[i] = id;
    rank[i] = atomicAdd(cell_cnt + id, 1);
}

// exclusive scan in tiles of 2048 (1024 threads x 2)
constexpr int kScanTile = 2048;

__device__ int block_excl_scan_1024(int v, int* warp_sums, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = warp_sums[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int incl = x + (w > 0 ? warp_sums[w - 1] : 0);
    *total = warp_sums[31];
    __syncthreads();
    return incl - v;
}

__global__ void __launch_bounds__(1024) k_scan_tiles(const int* __restrict__ in, int n,
                                                     int* __restrict__ out, int* tile_sum) {
    __shared__ int ws[32];
    const int base = blockIdx.x * kScanTile;
    const int i0 = base + 2 * threadIdx.x;
    const int v0 = i0 < n ? in[i0] : 0;
    const int v1 = i0 + 1 < n ? in[i0 + 1] : 0;
    int total;
    const int ex = block_excl_scan_1024(v0 + v1, ws, &total);
    if (i0 < n) out[i0] = ex;
    if (i0 + 1 < n) out[i0 + 1] = ex + v0;
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int* tile_sum, int ntiles, int* grand) {
    __shared__ int ws[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < ntiles; base += 1024) {
        const int t = base + threadIdx.x;
        const int v = t < ntiles ? tile_sum[t] : 0;
        int total;
        const int ex = block_excl_scan_1024(v, ws, &total);
        if (t < ntiles) tile_sum[t] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = carry;
}

__global__ void k_scan_add(int* out, int n, const int* tile_sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_sum[i / kScanTile];
}

__global__ void k_fill(const int* __restrict__ cell_of, const int* __restrict__ rank,
                       const int* __restrict__ cell_start, int N, int* cell_atoms) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    cell_atoms[cell_start[cell_of[i]] + rank[i]] = i;
}

// order each cell's atoms by index so that lists do not depend on the order
// in which atomics handed out ranks, then write the positions in that order
// (x, y, z, atom index as bits): the list build reads a row's candidates as
// one contiguous range, with no dependent index load
__global__ void k_sort_cells(const int* __restrict__ cell_start, int ncell, int* cell_atoms,
                             const float4* __restrict__ pos4, float4* __restrict__ cell_pos) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    const int s0 = cell_start[c], s1 = cell_start[c + 1];
    for (int a = s0 + 1; a < s1; ++a) {
        const int v = cell_atoms[a];
        int b = a - 1;
        while (b >= s0 && cell_atoms[b] > v) {
            cell_atoms[b + 1] = cell_atoms[b];
            --b;
        }
        cell_atoms[b + 1] = v;
    }
    for (int a = s0; a < s1; ++a) {
        const int j = cell_atoms[a];
        const float4 q = pos4[j];
        cell_pos[a] = make_float4(q.x, q.y, q.z, i2f(j));
    }
}

__device__ __forceinline__ int floor_div(int a, int b) {
    int q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

// One pass over the stencil.  The list is written in three groups:
// [d < rc_ang + skin] (the angular prefix) | [d < rc_rad] | [rc_rad <= d <
// rc_rad + skin].  Angular candidates fill it from slot 0 up, radial ones
// inside rc_rad from slot cap-1 down, the shell beyond rc_rad goes to a
// scratch buffer; at the end the downward block is reversed and moved behind
// the prefix and the shell appended, all in visit order.  With the pairs
// inside the cutoff first, a warp's late iterations are mostly outside the
// cutoff for all of its lanes and skip the pair work together.
//
// The stencil is visited row by row: for each (ox, oy) the cells oz =
// -half..half are consecutive cell ids (one range of the cell-ordered
// positions, which carry the atom index) except where they wrap around the
// box, which splits the row in two ranges with different z images.  The
// visit order is that of the cell triple loop.  For the reverse-slot search
// the kernel also records, per atom, where each row's angular entries start
// (row_start) and, per angular slot, its row.
__global__ void __launch_bounds__(128) k_build(const float4* __restrict__ pos4,
                                               const int* __restrict__ cfg,
                                               const float* __restrict__ box,
                                               const CellPlan* __restrict__ plan,
                                               const int* __restrict__ cell_of,
                                               const int* __restrict__ cell_start,
                                               const float4* __restrict__ cell_pos, int N,
                                               float rc2_rad, float rc2_ang, float rc2_phys,
                                               int2* __restrict__ shell, unsigned char* __restrict__ row_start,
                                               unsigned char* __restrict__ slot_row, nep_nlist nl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = cfg[i];
    const CellPlan p = plan[b];
    const float L[3] = {box[3 * b], box[3 * b + 1], box[3 * b + 2]};
    const float4 pi = pos4[i];
    int c = cell_of[i] - p.base;
    const int cz = c % p.nc[2];
    c /= p.nc[2];
    const int cy = c % p.nc[1];
    const int cx = c / p.nc[1];
    int n_ang = 0, n_in = 0, n_out = 0, w_ang = 0;
    const int cap = nl.cap, cap_ang = nl.cap_ang;
    const int rows = (2 * p.half[0] + 1) * (2 * p.half[1] + 1);
    const bool track = rows <= kMaxRows && cap_ang < 256;
    unsigned char* rs = row_start + (size_t)i * kRowStride;
    // Cells that cannot hold a candidate are skipped: for each stencil row
    // the z range shrinks to the cells that meet the sphere of the list
    // cutoff (plus a margin far above the rounding of the binning) around
    // atom i, given the row's distance from i in x and y.  Skipping only
    // cells whose every point is beyond the cutoff leaves the list, its
    // order and the row starts unchanged.
    const float cs[3] = {L[0] / (float)p.nc[0], L[1] / (float)p.nc[1], L[2] / (float)p.nc[2]};
    const float rl = sqrtf(rc2_rad) + kPruneMargin;
    const float rl2 = rl * rl;
    int row = 0;
    for (int ox = -p.half[0]; ox <= p.half[0]; ++ox) {
        const int ux = cx + ox, sx = floor_div(ux, p.nc[0]), wx = ux - sx * p.nc[0];
        const float gx = fmaxf(fmaxf((float)ux * cs[0] - pi.x, pi.x - (float)(ux + 1) * cs[0]), 0.0f);
        for (int oy = -p.half[1]; oy <= p.half[1]; ++oy, ++row) {
            const int uy = cy + oy, sy = floor_div(uy, p.nc[1]), wy = uy - sy * p.nc[1];
            if (track) rs[row] = (unsigned char)(n_ang < 255 ? n_ang : 255);
            const float fx = mul_rn((float)sx, L[0]);
            const float fy = mul_rn((float)sy, L[1]);
            const int rowcell = p.base + (wx * p.nc[1] + wy) * p.nc[2];
            const float gy = fmaxf(fmaxf((float)uy * cs[1] - pi.y, pi.y - (float)(uy + 1) * cs[1]), 0.0f);
            const float rem = rl2 - gx * gx - gy * gy;
            // z range [cz - half, cz + half] cut to the cells that meet the
            // sphere, in pieces of one z image each
            int lo = cz - p.half[2];
            int hi = cz + p.half[2];
            if (rem <= 0.0f) {
                hi = lo - 1;
            } else {
                const float hz = sqrtf(rem);
                lo = max(lo, (int)floorf((pi.z - hz) / cs[2]));
                hi = min(hi, (int)floorf((pi.z + hz) / cs[2]));
            }
            while (lo <= hi) {
                const int sz = floor_div(lo, p.nc[2]);
                const int seg_hi = min(hi, (sz + 1) * p.nc[2] - 1);
                const int wz0 = lo - sz * p.nc[2], wz1 = seg_hi - sz * p.nc[2];
                lo = seg_hi + 1;
                const float fz = mul_rn((float)sz, L[2]);
                const bool zero_img = (sx == 0 && sy == 0 && sz == 0);
                const int sh = pack_shift(sx, sy, sz);
                const int q0 = cell_start[rowcell + wz0], q1 = cell_start[rowcell + wz1 + 1];
                // candidates one ahead
                float4 c_nx = q0 < q1 ? cell_pos[q0] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                for (int q = q0; q < q1; ++q) {
                    const float4 pj = c_nx;
                    if (q + 1 < q1) c_nx = cell_pos[q + 1];
                    const int j = f2i(pj.w);
                    if (j == i && zero_img) continue;
                    const float dx = add_rn(sub_rn(pj.x, pi.x), fx);
                    const float dy = add_rn(sub_rn(pj.y, pi.y), fy);
                    const float dz = add_rn(sub_rn(pj.z, pi.z), fz);
                    const float d2 = dist2(dx, dy, dz);
                    if (!(d2 < rc2_rad)) continue;
                    // the angular and the inside entries share one store
                    // path (slots from the bottom and from the top)
                    const bool ang = d2 < rc2_ang;
                    if (ang || d2 < rc2_phys) {
                        int slot;
                        if (ang) {
                            slot = n_ang < cap_ang && n_ang + n_in < cap ? n_ang : -1;
                            ++n_ang;
                            if (slot >= 0) w_ang = n_ang;
                        } else {
                            slot = n_ang + n_in < cap ? cap - 1 - n_in : -1;
                            ++n_in;
                        }
                        if (slot >= 0) {
                            const size_t at = (size_t)slot * N + i;
                            nl.nbr[at] = j;
                            if (nl.shift) nl.shift[at] = sh;
                            if (ang && track) slot_row[at] = (unsigned char)row;
                        }
                    } else {
                        if (n_out < cap) shell[(size_t)n_out * N + i] = make_int2(j, sh);
                        ++n_out;
                    }
                }
            }
        }
    }
    if (track) rs[rows] = (unsigned char)(n_ang < 255 ? n_ang : 255);
    const int n_rest = n_in + n_out;
    const int n_total = n_ang + n_rest;
    const bool over = n_total > cap || n_ang > cap_ang;
    if (over) {
        set_flag(nl.status, 0);
        atomicMax(nl.status + 1, n_total);
        atomicMax(nl.status + 2, n_ang);
        // only the contiguous angular prefix that was written is kept
        nl.cnt[i] = w_ang;
        nl.cnt_ang[i] = w_ang;
        return;
    }
    // the inside block sits reversed at [cap - n_in, cap).  Where it does not
    // overlap its target behind the prefix it is copied there in reverse
    // order; otherwise it is reversed in place, then copied down (ascending
    // copy, target never above source).  Then the shell is appended.
    const int base = cap - n_in;
    if (base >= n_ang + n_in) {
        for (int k = 0; k < n_in; ++k) {
            const size_t from = (size_t)(cap - 1 - k) * N + i, to = (size_t)(n_ang + k) * N + i;
            nl.nbr[to] = nl.nbr[from];
            if (nl.shift) nl.shift[to] = nl.shift[from];
        }
    } else {
        for (int k = 0; k < n_in / 2; ++k) {
            const size_t x = (size_t)(base + k) * N + i, y = (size_t)(cap - 1 - k) * N + i;
            const int t = nl.nbr[x];
            nl.nbr[x] = nl.nbr[y];
            nl.nbr[y] = t;
            if (nl.shift) {
                const int u = nl.shift[x];
                nl.shift[x] = nl.shift[y];
                nl.shift[y] = u;
            }
        }
        if (base != n_ang) {
            for (int k = 0; k < n_in; ++k) {
                const size_t from = (size_t)(base + k) * N + i, to = (size_t)(n_ang + k) * N + i;
                nl.nbr[to] = nl.nbr[from];
                if (nl.shift) nl.shift[to] = nl.shift[from];
            }
        }
    }
    for (int k = 0; k < n_out; ++k) {
        const int2 e = shell[(size_t)k * N + i];
        const size_t to = (size_t)(n_ang + n_in + k) * N + i;
        nl.nbr[to] = e.x;
        if (nl.shift) nl.shift[to] = e.y;
    }
    nl.cnt[i] = n_total;
    nl.cnt_ang[i] = n_ang;
}

// rev[s][i] = slot of i (with the opposite image) in the angular prefix of
// j = nbr[s][i].  j visits i in the mirrored stencil row, rows - 1 - row,
// so only that row's stretch of j's prefix is searched; stencils too large
// for the row table fall back to scanning j's whole prefix.
__global__ void k_rev(int N, const int* __restrict__ cfg, const CellPlan* __restrict__ plan,
                      const unsigned char* __restrict__ row_start, const unsigned char* __restrict__ slot_row,
                      nep_nlist nl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int na = nl.cnt_ang[i];
    const CellPlan p = plan[cfg[i]];
    const int rows = (2 * p.half[0] + 1) * (2 * p.half[1] + 1);
    const bool track = rows <= kMaxRows && nl.cap_ang < 256;
    for (int s = 0; s < na; ++s) {
        const int j = nl.nbr[(size_t)s * N + i];
        int want = 0;
        if (nl.shift) {
            int a, b, c;
            unpack_shift(nl.shift[(size_t)s * N + i], a, b, c);
            want = pack_shift(-a, -b, -c);
        }
        const int nj = nl.cnt_ang[j];
        int t0 = 0, t1 = nj;
        if (track) {
            const int mr = rows - 1 - (int)slot_row[(size_t)s * N + i];
            const unsigned char* rj = row_start + (size_t)j * kRowStride;
            t0 = rj[mr];
            t1 = min((int)rj[mr + 1], nj);
        }
        int found = -1;
        for (int t = t0; t < t1; ++t) {
            if (nl.nbr[(size_t)t * N + j] == i && (!nl.shift || nl.shift[(size_t)t * N + j] == want)) {
                found = t;
                break;
            }
        }
        if (found < 0) {
            set_flag(nl.status, 0);
            found = 0;
        }
        nl.rev[(size_t)s * N + i] = found;
    }
}

// ------------------------------------------------------------ optimiser
// one Adam step per parameter; c1 = lr / (1 - beta1^t), c2 = 1 / sqrt(1 - beta2^t)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float beta1, float beta2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float mk = beta1 * m[k] + (1.0f - beta1) * gk;
    const float vk = beta2 * v[k] + (1.0f - beta2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= c1 * mk / (sqrtf(vk) * c2 + eps);
}

// ------------------------------------------------------------ FP32 peak
// eight independent FMA chains per thread; a and b come from memory so that
// nothing folds, the sums are stored so that nothing is dropped
constexpr int kFmaIters = 4096;
__global__ void __launch_bounds__(256) k_fma_peak(const float* __restrict__ ab, float* __restrict__ out) {
    const float a = ab[0], b = ab[1];
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float sum = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) sum += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
}

// ------------------------------------------------------------ integrator
struct InvMass {
    float v[kMaxTypes];
};

__global__ void k_kick(float* __restrict__ vel, const float* __restrict__ force,
                       const int* __restrict__ type, InvMass im, int N, float half_dt,
                       float* __restrict__ pos, float dt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float s = half_dt * im.v[type[i] & (kMaxTypes - 1)];
    for (int d = 0; d < 3; ++d) {
        float v = vel[(size_t)d * N + i] + s * force[(size_t)d * N + i];
        vel[(size_t)d * N + i] = v;
        if (pos) pos[(size_t)d * N + i] += dt * v;
    }
}

// x wrapped into [0, L)
__device__ __forceinline__ float wrap_coord(float x, float L) {
    x = x - L * floorf(x / L);
    if (x >= L) x -= L;
    if (x < 0.0f) x += L;
    if (!(x < L)) x = 0.0f;
    return x;
}
__global__ void k_wrap(float* pos, const int* __restrict__ cfg, const float* __restrict__ box,
                       int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = cfg[i];
    for (int d = 0; d < 3; ++d) pos[(size_t)d * N + i] = wrap_coord(pos[(size_t)d * N + i], box[3 * b + d]);
}
// the same, with each atom's configuration found from the CSR offsets
__global__ void k_wrap_seg(float* pos, const int* __restrict__ atom_off, int B, const float* __restrict__ box,
                           int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int b = find_segment(atom_off, B, i);
    for (int d = 0; d < 3; ++d) pos[(size_t)d * N + i] = wrap_coord(pos[(size_t)d * N + i], box[3 * b + d]);
}

// ------------------------------------------------------------- loss adjoints
// Force residuals per chunk: lam_i = 2 wF (F_i - F_lbl,i) / (3 N_b B) and the
// FP64 partial sum of |dF|^2 (Eq. 20).
__global__ void __launch_bounds__(kRedThreads) k_loss_atoms(
    int N, int B, const int* __restrict__ atom_off, const int* __restrict__ chunk_start,
    const float* __restrict__ force, const float* __restrict__ f_lbl, float wF, float4* lam4,
    double* partial) {
    const int k = blockIdx.x;
    const int total = chunk_start[B];
    if (k >= total) return;
    const int b = find_segment(chunk_start, B, k);
    const int a0 = atom_off[b] + (k - chunk_start[b]) * kChunk;
    const int a1 = min(atom_off[b + 1], a0 + kChunk);
    const int nb = atom_off[b + 1] - atom_off[b];
    const float cf = 2.0f * wF / (3.0f * (float)nb * (float)B);
    double acc = 0.0;
    for (int i = a0 + threadIdx.x; i < a1; i += kRedThreads) {
        const float dx = force[i] - f_lbl[i];
        const float dy = force[N + i] - f_lbl[N + i];
        const float dz = force[2 * N + i] - f_lbl[2 * N + i];
        lam4[i] = make_float4(cf * dx, cf * dy, cf * dz, 0.0f);
        acc += (double)dx * dx + (double)dy * dy + (double)dz * dz;
    }
    __shared__ double red[kRedThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[k] = red[0];
}

// Per-configuration loss terms and energy/virial adjoints (Eqs. 18-21), and
// the batch loss summed in a fixed tree (one CTA).
__global__ void __launch_bounds__(kRedThreads) k_loss_cfg(
    int B, const int* __restrict__ atom_off, const int* __restrict__ chunk_start,
    const double* __restrict__ partial, const double* __restrict__ e_tot,
    const double* __restrict__ vir, const double* __restrict__ e_lbl,
    const double* __restrict__ v_lbl, float wE, float wF, float wV, int mode, float* aE, float* mu,
    double* loss) {
    // FP64 division is slow on this GPU: each configuration divides once,
    // by its atom count, and the rest are products
    const double iB = 1.0 / (double)B;
    double acc = 0.0;
    for (int b = threadIdx.x; b < B; b += kRedThreads) {
        const double nb = (double)(atom_off[b + 1] - atom_off[b]);
        const double n = nb > 0.0 ? nb : 1.0;
        const double in = 1.0 / n;
        double sF = 0.0;
        for (int k = chunk_start[b]; k < chunk_start[b + 1]; ++k) sF += partial[k];
        const double dE = e_tot[b] - e_lbl[b];
        double sV = 0.0;
        for (int c = 0; c < 9; ++c) {
            const double dv = vir[9 * b + c] - v_lbl[9 * b + c];
            sV += dv * dv;
        }
        constexpr double third = 1.0 / 3.0, ninth = 1.0 / 9.0;
        double Lb;
        if (mode == 0) {
            const double e = dE * in;
            Lb = wE * e * e + wF * sF * (third * in) + wV * sV * (ninth * in * in);
            aE[b] = (float)(2.0 * wE * dE * (in * in) * iB);
            const double fv = 2.0 * wV * (ninth * in * in) * iB;
            for (int c = 0; c < 9; ++c) mu[9 * b + c] = (float)(fv * (vir[9 * b + c] - v_lbl[9 * b + c]));
        } else {
            Lb = wE * dE * dE * in + wF * sF * (third * in) + wV * sV * (ninth * in);
            aE[b] = (float)(2.0 * wE * dE * in * iB);
            const double fv = 2.0 * wV * (ninth * in) * iB;
            for (int c = 0; c < 9; ++c) mu[9 * b + c] = (float)(fv * (vir[9 * b + c] - v_lbl[9 * b + c]));
        }
        if (nb > 0.0) acc += Lb;
    }
    __shared__ double red[kRedThreads];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kRedThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) *loss = red[0] * iB;
}

// External adjoints (vector-Jacobian product) into the kernels' layout.
__global__ void k_pack_adjoint(int N, int B, const float* __restrict__ lam,
                               const double* __restrict__ a_e, const double* __restrict__ mu_in,
                               float4* lam4, float* aE, float* mu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) lam4[i] = make_float4(lam[i], lam[N + i], lam[2 * N + i], 0.0f);
    if (i < B) {
        aE[i] = (float)a_e[i];
        for (int c = 0; c < 9; ++c) mu[9 * i + c] = (float)mu_in[9 * i + c];
    }
}

inline int blocks(int n, int t) { return (n + t - 1) / t; }

}  // namespace

// ------------------------------------------------------------ launchers
cudaError_t launch_pack(const float* pos, const int* type, const int* atom_off, int N, int B,
                        int T, float4* pos4, int* cfg, int* status, cudaStream_t st) {
    if (N > 0) k_pack<<<blocks(N, 256), 256, 0, st>>>(pos, type, atom_off, N, B, T, pos4, cfg, status);
    return cudaGetLastError();
}

cudaError_t launch_chunk_plan(const int* atom_off, int B, int* chunk_start, cudaStream_t st) {
    k_chunk_plan<<<1, 1024, 0, st>>>(atom_off, B, chunk_start);
    return cudaGetLastError();
}

cudaError_t launch_chunk_reduce(const EvalArgs& a, const FinishArgs& f, int max_chunks, cudaStream_t st) {
    if (max_chunks > 0) k_chunk_reduce<<<max_chunks, kRedThreads, 0, st>>>(a, f);
    return cudaGetLastError();
}

cudaError_t launch_final_reduce(int B, const int* chunk_start, const double* partial,
                                double* e_tot, double* virial, cudaStream_t st) {
    if (B > 0) k_final_reduce<<<B, kRedThreads, 0, st>>>(B, chunk_start, partial, e_tot, virial);
    return cudaGetLastError();
}

size_t nbr_cell_capacity(int N, int B) { return 2 * (size_t)N + 27 * (size_t)B; }

cudaError_t launch_neighbors(const float* pos, const float4* pos4, const int* atom_off, const float* box,
                             const int* cfg, int N, int B, float rc_list, float rc_list_ang, float rc_phys,
                             int min_image, nep_nlist* nl, const NbrWork& w, cudaStream_t st) {
    cudaError_t e;
    (void)min_image;
    if (N == 0) return cudaSuccess;
    const int cmax = w.cmax;
    k_cell_plan<<<blocks(B, 128), 128, 0, st>>>(box, atom_off, B, rc_list, w.plan, nl->status);
    k_plan_scan<<<1, 32, 0, st>>>(w.plan, B);
    if ((e = cudaMemsetAsync(w.cell_cnt, 0, sizeof(int) * (size_t)(cmax + 1), st)) != cudaSuccess)
        return e;
    k_bin<<<blocks(N, 256), 256, 0, st>>>(pos, cfg, box, w.plan, N, w.cell_of, w.rank, w.cell_cnt,
                                          nl->status);
    const int n = cmax + 1;
    const int ntiles = blocks(n, kScanTile);
    k_scan_tiles<<<ntiles, 1024, 0, st>>>(w.cell_cnt, n, w.cell_start, w.scan_tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(w.scan_tmp, ntiles, w.scan_tmp + ntiles);
    k_scan_add<<<blocks(n, 256), 256, 0, st>>>(w.cell_start, n, w.scan_tmp);
    k_fill<<<blocks(N, 256), 256, 0, st>>>(w.cell_of, w.rank, w.cell_start, N, w.cell_atoms);
    k_sort_cells<<<blocks(cmax, 128), 128, 0, st>>>(w.cell_start, cmax, w.cell_atoms, pos4, w.cell_pos);
    const float rr = rc_list * rc_list, ra = rc_list_ang * rc_list_ang, rp = rc_phys * rc_phys;
    k_build<<<blocks(N, 128), 128, 0, st>>>(pos4, cfg, box, w.plan, w.cell_of, w.cell_start,
                                            w.cell_pos, N, rr, ra, rp, w.shell, w.row_start, w.slot_row, *nl);
    k_rev<<<blocks(N, 128), 128, 0, st>>>(N, cfg, w.plan, w.row_start, w.slot_row, *nl);
    return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, int n, float beta1, float beta2,
                        float eps, float c1, float c2, cudaStream_t st) {
    if (n > 0) k_adam<<<blocks(n, 256), 256, 0, st>>>(p, g, m, v, n, beta1, beta2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t fp32_peak(cudaStream_t st, double* tflops) {
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev))) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev))) return e;
    const int blocks_n = nsm * 8, threads = 256;
    float* buf = nullptr;
    if ((e = cudaMalloc(&buf, sizeof(float) * ((size_t)blocks_n * threads + 2)))) return e;
    const float ab[2] = {0.999f, 1e-3f};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f, best = 1e30f;
    if (!(e = cudaMemcpyAsync(buf, ab, sizeof ab, cudaMemcpyHostToDevice, st)) && !(e = cudaEventCreate(&e0)) &&
        !(e = cudaEventCreate(&e1))) {
        for (int r = 0; r < 4 && !e; ++r) {
            cudaEventRecord(e0, st);
            k_fma_peak<<<blocks_n, threads, 0, st>>>(buf, buf + 2);
            cudaEventRecord(e1, st);
            if (!(e = cudaEventSynchronize(e1)) && !(e = cudaEventElapsedTime(&ms, e0, e1)) && r > 0 && ms < best)
                best = ms;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(buf);
    if (e) return e;
    *tflops = 2.0 * 8.0 * kFmaIters * (double)blocks_n * threads / (best * 1e-3) / 1e12;
    return cudaGetLastError();
}

cudaError_t launch_kick(float* vel, const float* force, const int* type, const float* inv_mass,
                        int N, float half_dt, float* pos, float dt, cudaStream_t st) {
    InvMass im;
    for (int t = 0; t < kMaxTypes; ++t) im.v[t] = inv_mass[t];
    if (N > 0) k_kick<<<blocks(N, 256), 256, 0, st>>>(vel, force, type, im, N, half_dt, pos, dt);
    return cudaGetLastError();
}

cudaError_t launch_loss(int N, int B, const int* atom_off, const int* chunk_start, int max_chunks,
                        const float* force, const float* f_lbl, const double* e_tot,
                        const double* vir, const double* e_lbl, const double* v_lbl,
                        const float* w, int mode, float4* lam4, float* aE, float* mu,
                        double* partial, double* loss, cudaStream_t st) {
    if (max_chunks > 0)
        k_loss_atoms<<<max_chunks, kRedThreads, 0, st>>>(N, B, atom_off, chunk_start, force, f_lbl, w[1],
                                                         lam4, partial);
    k_loss_cfg<<<1, kRedThreads, 0, st>>>(B, atom_off, chunk_start, partial, e_tot, vir, e_lbl, v_lbl,
                                          w[0], w[1], w[2], mode, aE, mu, loss);
    return cudaGetLastError();
}

cudaError_t launch_pack_adjoint(int N, int B, const float* lam, const double* a_e, const double* mu_in,
                                float4* lam4, float* aE, float* mu, cudaStream_t st) {
    const int n = N > B ? N : B;
    if (n > 0) k_pack_adjoint<<<blocks(n, 256), 256, 0, st>>>(N, B, lam, a_e, mu_in, lam4, aE, mu);
    return cudaGetLastError();
}

cudaError_t launch_wrap(float* pos, const int* cfg, const float* box, int N, cudaStream_t st) {
    if (N > 0) k_wrap<<<blocks(N, 256), 256, 0, st>>>(pos, cfg, box, N);
    return cudaGetLastError();
}

cudaError_t launch_wrap_segments(float* pos, const int* atom_off, int B, const float* box, int N, cudaStream_t st) {
    if (N > 0) k_wrap_seg<<<blocks(N, 256), 256, 0, st>>>(pos, atom_off, B, box, N);
    return cudaGetLastError();
}

}  // namespace nep
