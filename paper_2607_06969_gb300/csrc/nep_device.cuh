// Device math of the NEP pair terms: cutoff and Chebyshev basis (Eqs. 12-15),
// real solid harmonics for l = 1..4 (Eq. 16) and their gradients.
#pragma once
#include "nep_internal.h"

#if !defined(__CUDA_ARCH__)
#include <cmath>
#endif

namespace nep {

// IEEE single operations that the compiler must not contract into FMAs;
// the neighbour predicate and the pair vectors are defined with them.
NEP_HD float add_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    volatile float r = a + b;
    return r;
#endif
}
NEP_HD float mul_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    volatile float r = a * b;
    return r;
#endif
}
NEP_HD float sub_rn(float a, float b) {
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    volatile float r = a - b;
    return r;
#endif
}
// correctly rounded reciprocal
NEP_HD float rcp_f(float x) {
#if defined(__CUDA_ARCH__)
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}
NEP_HD float tanh_f(float x) {
#if defined(__CUDA_ARCH__)
    return tanhf(x);
#else
    return (float)std::tanh((double)x);
#endif
}
NEP_HD float sqrt_f(float x) {
#if defined(__CUDA_ARCH__)
    return sqrtf(x);
#else
    return (float)std::sqrt((double)x);
#endif
}
// Distance r and 1/r of a pair from d2 = |r_ij|^2 > 0: one reciprocal
// square root (rsqrtf, within 2 ulp) and a product on the device, in place
// of a correctly rounded square root and reciprocal (2.8% of an evaluation
// at 900k atoms, measured; the results stay within the FP32 parity bars).
NEP_HD void dist_rinv(float d2, float& r, float& ir) {
#if defined(__CUDA_ARCH__)
    ir = rsqrtf(d2);
    r = d2 * ir;
#else
    r = sqrt_f(d2);
    ir = rcp_f(r);
#endif
}
NEP_HD float dist_r(float d2) {
#if defined(__CUDA_ARCH__)
    return d2 * rsqrtf(d2);
#else
    return sqrt_f(d2);
#endif
}
NEP_HD float rint_f(float x) {
#if defined(__CUDA_ARCH__)
    return rintf(x);
#else
    return std::nearbyint(x);
#endif
}
// eight consecutive floats from a 32-byte aligned global address that no
// thread writes during the kernel: one 256-bit load on the device
NEP_HD void load8_ro(const float* p, float* v) {
#if defined(__CUDA_ARCH__)
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
        : "l"(p));
#else
    for (int k = 0; k < 8; ++k) v[k] = p[k];
#endif
}

// Two independent FP32 FMAs in one paired instruction on the device
// (a.x * b.x + c.x, a.y * b.y + c.y, each rounded once as fmaf rounds it):
// pairing two accumulation chains leaves every result bit unchanged and
// halves the instructions the chains issue.
NEP_HD float2 ffma2(float2 a, float2 b, float2 c) {
#if defined(__CUDA_ARCH__)
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

// index of the lowest set bit of a non-zero word
NEP_HD int low_bit(unsigned long long m) {
#if defined(__CUDA_ARCH__)
    return __ffsll((long long)m) - 1;
#else
    return __builtin_ctzll(m);
#endif
}
NEP_HD int f2i(float x) {
#if defined(__CUDA_ARCH__)
    return __float_as_int(x);
#else
    int r; memcpy(&r, &x, 4); return r;
#endif
}
NEP_HD float i2f(int x) {
#if defined(__CUDA_ARCH__)
    return __int_as_float(x);
#else
    float r; memcpy(&r, &x, 4); return r;
#endif
}

// Packed image shift: int8 sx | sy << 8 | sz << 16.
NEP_HD int pack_shift(int sx, int sy, int sz) {
    return (sx & 0xff) | ((sy & 0xff) << 8) | ((sz & 0xff) << 16);
}
NEP_HD void unpack_shift(int v, int& sx, int& sy, int& sz) {
    sx = (int)(signed char)(v & 0xff);
    sy = (int)(signed char)((v >> 8) & 0xff);
    sz = (int)(signed char)((v >> 16) & 0xff);
}

// Pair vector r_ij = (x_j - x_i) + s * L with the list's image, or with the
// minimum image when the list carries no shifts.  Same operation order as the
// neighbour predicate.
NEP_HD void pair_vector(float4 pi, float4 pj, float Lx, float Ly, float Lz, float iLx, float iLy,
                        float iLz, int min_image, int packed, float& dx, float& dy, float& dz) {
    float ux = sub_rn(pj.x, pi.x), uy = sub_rn(pj.y, pi.y), uz = sub_rn(pj.z, pi.z);
    float sx, sy, sz;
    if (min_image) {
        sx = -rint_f(ux * iLx);
        sy = -rint_f(uy * iLy);
        sz = -rint_f(uz * iLz);
    } else {
        int a, b, c;
        unpack_shift(packed, a, b, c);
        sx = (float)a; sy = (float)b; sz = (float)c;
    }
    dx = add_rn(ux, mul_rn(sx, Lx));
    dy = add_rn(uy, mul_rn(sy, Ly));
    dz = add_rn(uz, mul_rn(sz, Lz));
}

NEP_HD float dist2(float dx, float dy, float dz) {
    return add_rn(add_rn(mul_rn(dx, dx), mul_rn(dy, dy)), mul_rn(dz, dz));
}

// cos(pi z) and sin(pi z) for z = r/rc in [0, 1): with w = z - 1/2,
// cos(pi z) = -sin(pi w) and sin(pi z) = cos(pi w), |pi w| <= pi/2, summed
// as their Taylor series in y = (pi w)^2 (Horner), through y^6: the first
// omitted terms are below (pi/2)^15/15! = 6.7e-10 and (pi/2)^14/14! = 6.9e-9,
// under the FP32 rounding of the result.
NEP_HD void cutoff_trig(float z, float& c, float& s) {
    // pi w with pi split in two floats, so that the product keeps ~45 bits
    const float w = z - 0.5f;
    const float t = fmaf(3.14159274101257324f, w, -8.74227766e-8f * w);
    const float y = t * t;
    float ps = 1.0f / 6227020800.0f;                 // 1/13!
    ps = fmaf(ps, y, -1.0f / 39916800.0f);            // 1/11!
    ps = fmaf(ps, y, 1.0f / 362880.0f);               // 1/9!
    ps = fmaf(ps, y, -1.0f / 5040.0f);                // 1/7!
    ps = fmaf(ps, y, 1.0f / 120.0f);
    ps = fmaf(ps, y, -1.0f / 6.0f);
    ps = fmaf(ps, y, 1.0f);
    float pc = 1.0f / 479001600.0f;                  // 1/12!
    pc = fmaf(pc, y, -1.0f / 3628800.0f);             // 1/10!
    pc = fmaf(pc, y, 1.0f / 40320.0f);                // 1/8!
    pc = fmaf(pc, y, -1.0f / 720.0f);
    pc = fmaf(pc, y, 1.0f / 24.0f);
    pc = fmaf(pc, y, -0.5f);
    pc = fmaf(pc, y, 1.0f);
    c = -t * ps;
    s = pc;
}

// Q_k(r) = (T_k(x)+1)/2 f_c(r), x = 2(r/rc-1)^2-1, f_c = (1+cos(pi r/rc))/2.
template <int K>
NEP_HD void basis(float r, float inv_rc, float* f) {
    float cz, sz;
    cutoff_trig(r * inv_rc, cz, sz);
    float fc2 = 0.25f * (1.0f + cz);                       // f_c / 2
    float t = r * inv_rc - 1.0f;
    float x = 2.0f * t * t - 1.0f;
    float Tm = 1.0f, Tk = x;
    f[0] = 2.0f * fc2;
    if (K > 1) f[1] = (x + 1.0f) * fc2;
#pragma unroll
    for (int k = 2; k < K; ++k) {
        float Tn = 2.0f * x * Tk - Tm;
        f[k] = (Tn + 1.0f) * fc2;
        Tm = Tk;
        Tk = Tn;
    }
}

// Q_k and dQ_k/dr.  T'_{k+1} = 2 T_k + 2x T'_k - T'_{k-1}.
template <int K>
NEP_HD void basis_d(float r, float inv_rc, float* f, float* fp) {
    float sp, cp;
    cutoff_trig(r * inv_rc, cp, sp);
    float fc2 = 0.25f * (1.0f + cp);
    float dfc2 = (-0.25f * 3.14159265358979f) * inv_rc * sp;
    float t = r * inv_rc - 1.0f;
    float x = 2.0f * t * t - 1.0f;
    float dxdr = 4.0f * t * inv_rc;
    float a = dxdr * fc2;
    float Tm = 1.0f, Tk = x, dTm = 0.0f, dTk = 1.0f;
    f[0] = 2.0f * fc2;
    fp[0] = 2.0f * dfc2;
    if (K > 1) {
        f[1] = (x + 1.0f) * fc2;
        fp[1] = a + (x + 1.0f) * dfc2;
    }
#pragma unroll
    for (int k = 2; k < K; ++k) {
        float Tn = 2.0f * x * Tk - Tm;
        float dTn = 2.0f * Tk + 2.0f * x * dTk - dTm;
        f[k] = (Tn + 1.0f) * fc2;
        fp[k] = dTn * a + (Tn + 1.0f) * dfc2;
        Tm = Tk; Tk = Tn; dTm = dTk; dTk = dTn;
    }
}

// Weights C_lm such that sum_m C_lm P_lm(a) P_lm(b) = P_l(a.b) for unit a, b,
// i.e. 4 pi/(2l+1) times the squared normalisation of each real harmonic.
NEP_HD float clm(int lm) {
    switch (lm) {
        case 0: case 1: case 2: return 1.0f;
        case 3: case 4: case 6: return 3.0f;
        case 5: return 0.25f;
        case 7: return 0.75f;
        case 8: case 14: return 0.625f;
        case 9: return 15.0f;
        case 10: case 12: return 0.375f;
        case 11: return 0.25f;
        case 13: return 3.75f;
        case 15: return 8.75f;
        case 16: case 22: return 4.375f;
        case 17: return 1.25f;
        case 18: case 20: return 0.625f;
        case 19: return 1.0f / 64.0f;
        case 21: return 0.3125f;
        default: return 35.0f / 64.0f;   // 23
    }
}
NEP_HD int lm_l(int lm) { return lm < 3 ? 1 : (lm < 8 ? 2 : (lm < 15 ? 3 : 4)); }

// Real solid harmonics P_lm(u) of a unit vector (homogeneous polynomials of
// degree l evaluated on the unit sphere), order as in clm().
NEP_HD void harmonics(float x, float y, float z, float* Y) {
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    Y[0] = y; Y[1] = z; Y[2] = x;
    Y[3] = xy; Y[4] = yz; Y[5] = 3.0f * zz - 1.0f; Y[6] = xz; Y[7] = xx - yy;
    float a5 = 5.0f * zz - 1.0f;
    Y[8] = y * (3.0f * xx - yy);
    Y[9] = xy * z;
    Y[10] = y * a5;
    Y[11] = z * (5.0f * zz - 3.0f);
    Y[12] = x * a5;
    Y[13] = z * (xx - yy);
    Y[14] = x * (xx - 3.0f * yy);
    float b7 = 7.0f * zz - 1.0f, c7 = 7.0f * zz - 3.0f;
    Y[15] = xy * (xx - yy);
    Y[16] = yz * (3.0f * xx - yy);
    Y[17] = xy * b7;
    Y[18] = yz * c7;
    Y[19] = (35.0f * zz - 30.0f) * zz + 3.0f;
    Y[20] = xz * c7;
    Y[21] = (xx - yy) * b7;
    Y[22] = xz * (xx - 3.0f * yy);
    Y[23] = xx * (xx - 3.0f * yy) - yy * (3.0f * xx - yy);
}

// Component m of the real solid harmonics: value P_m(u) on the unit sphere
// and the gradient of the homogeneous polynomial at u.  With m a
// compile-time constant the switch folds away.
template <class R>
struct HarmTermsT {
    R x, y, z, xx, yy, zz, xy, xz, yz;
};
using HarmTerms = HarmTermsT<float>;
template <class R>
NEP_HD HarmTermsT<R> harm_terms(R x, R y, R z) {
    HarmTermsT<R> t;
    t.x = x; t.y = y; t.z = z;
    t.xx = x * x; t.yy = y * y; t.zz = z * z;
    t.xy = x * y; t.xz = x * z; t.yz = y * z;
    return t;
}
template <class R>
NEP_HD void harm_m(int m, const HarmTermsT<R>& t, R& Y, R& gx, R& gy, R& gz) {
    const R x = t.x, y = t.y, z = t.z, xx = t.xx, yy = t.yy, zz = t.zz;
    const R xy = t.xy, xz = t.xz, yz = t.yz;
    switch (m) {
        case 0: Y = y; gx = R(0.0); gy = R(1.0); gz = R(0.0); break;
        case 1: Y = z; gx = R(0.0); gy = R(0.0); gz = R(1.0); break;
        case 2: Y = x; gx = R(1.0); gy = R(0.0); gz = R(0.0); break;
        case 3: Y = xy; gx = y; gy = x; gz = R(0.0); break;
        case 4: Y = yz; gx = R(0.0); gy = z; gz = y; break;
        case 5: Y = R(3.0) * zz - R(1.0); gx = -R(2.0) * x; gy = -R(2.0) * y; gz = R(4.0) * z; break;
        case 6: Y = xz; gx = z; gy = R(0.0); gz = x; break;
        case 7: Y = xx - yy; gx = R(2.0) * x; gy = -R(2.0) * y; gz = R(0.0); break;
        case 8: Y = y * (R(3.0) * xx - yy); gx = R(6.0) * xy; gy = R(3.0) * (xx - yy); gz = R(0.0); break;
        case 9: Y = xy * z; gx = yz; gy = xz; gz = xy; break;
        case 10: Y = y * (R(5.0) * zz - R(1.0)); gx = -R(2.0) * xy; gy = R(4.0) * zz - xx - R(3.0) * yy; gz = R(8.0) * yz; break;
        case 11: Y = z * (R(5.0) * zz - R(3.0)); gx = -R(6.0) * xz; gy = -R(6.0) * yz; gz = R(6.0) * zz - R(3.0) * xx - R(3.0) * yy; break;
        case 12: Y = x * (R(5.0) * zz - R(1.0)); gx = R(4.0) * zz - R(3.0) * xx - yy; gy = -R(2.0) * xy; gz = R(8.0) * xz; break;
        case 13: Y = z * (xx - yy); gx = R(2.0) * xz; gy = -R(2.0) * yz; gz = xx - yy; break;
        case 14: Y = x * (xx - R(3.0) * yy); gx = R(3.0) * (xx - yy); gy = -R(6.0) * xy; gz = R(0.0); break;
        case 15: Y = xy * (xx - yy); gx = y * (R(3.0) * xx - yy); gy = x * (xx - R(3.0) * yy); gz = R(0.0); break;
        case 16: Y = yz * (R(3.0) * xx - yy); gx = R(6.0) * xy * z; gy = R(3.0) * z * (xx - yy); gz = y * (R(3.0) * xx - yy); break;
        case 17: Y = xy * (R(7.0) * zz - R(1.0)); gx = -y * (R(3.0) * xx + yy - R(6.0) * zz); gy = -x * (xx + R(3.0) * yy - R(6.0) * zz); gz = R(12.0) * xy * z; break;
        case 18: Y = yz * (R(7.0) * zz - R(3.0)); gx = -R(6.0) * xy * z; gy = -z * (R(3.0) * xx + R(9.0) * yy - R(4.0) * zz); gz = -R(3.0) * y * (xx + yy - R(4.0) * zz); break;
        case 19: Y = (R(35.0) * zz - R(30.0)) * zz + R(3.0); gx = R(12.0) * x * (xx + yy - R(4.0) * zz); gy = R(12.0) * y * (xx + yy - R(4.0) * zz); gz = -R(16.0) * z * (R(3.0) * xx + R(3.0) * yy - R(2.0) * zz); break;
        case 20: Y = xz * (R(7.0) * zz - R(3.0)); gx = -z * (R(9.0) * xx + R(3.0) * yy - R(4.0) * zz); gy = -R(6.0) * xy * z; gz = -R(3.0) * x * (xx + yy - R(4.0) * zz); break;
        case 21: Y = (xx - yy) * (R(7.0) * zz - R(1.0)); gx = -R(4.0) * x * (xx - R(3.0) * zz); gy = R(4.0) * y * (yy - R(3.0) * zz); gz = R(12.0) * z * (xx - yy); break;
        case 22: Y = xz * (xx - R(3.0) * yy); gx = R(3.0) * z * (xx - yy); gy = -R(6.0) * xy * z; gz = x * (xx - R(3.0) * yy); break;
        default: Y = xx * (xx - R(3.0) * yy) - yy * (R(3.0) * xx - yy); gx = R(4.0) * x * (xx - R(3.0) * yy); gy = -R(4.0) * y * (R(3.0) * xx - yy); gz = R(0.0); break;
    }
}

// g = sum_lm a_lm grad P_lm(u) (gradient of the homogeneous polynomials).
NEP_HD void harmonics_grad_contract(float x, float y, float z, const float* a, float& gx,
                                    float& gy, float& gz) {
    float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    float xyz = xy * z;
    // l = 1
    gx = a[2];
    gy = a[0];
    gz = a[1];
    // l = 2
    gx += a[3] * y - 2.0f * a[5] * x + a[6] * z + 2.0f * a[7] * x;
    gy += a[3] * x + a[4] * z - 2.0f * a[5] * y - 2.0f * a[7] * y;
    gz += a[4] * y + 4.0f * a[5] * z + a[6] * x;
    // l = 3
    float d3 = 3.0f * (xx - yy);
    gx += a[8] * 6.0f * xy + a[9] * yz - a[10] * 2.0f * xy - a[11] * 6.0f * xz
          + a[12] * (4.0f * zz - 3.0f * xx - yy) + a[13] * 2.0f * xz + a[14] * d3;
    gy += a[8] * d3 + a[9] * xz + a[10] * (4.0f * zz - xx - 3.0f * yy) - a[11] * 6.0f * yz
          - a[12] * 2.0f * xy - a[13] * 2.0f * yz - a[14] * 6.0f * xy;
    gz += a[9] * xy + a[10] * 8.0f * yz + a[11] * (6.0f * zz - 3.0f * xx - 3.0f * yy)
          + a[12] * 8.0f * xz + a[13] * (xx - yy);
    // l = 4
    float e1 = 3.0f * xx - yy, e2 = xx - 3.0f * yy, e3 = xx + yy - 4.0f * zz;
    gx += a[15] * y * e1 + a[16] * 6.0f * xyz - a[17] * y * (3.0f * xx + yy - 6.0f * zz)
          - a[18] * 6.0f * xyz + a[19] * 12.0f * x * e3 - a[20] * z * (9.0f * xx + 3.0f * yy - 4.0f * zz)
          - a[21] * 4.0f * x * (xx - 3.0f * zz) + a[22] * 3.0f * z * (xx - yy) + a[23] * 4.0f * x * e2;
    gy += a[15] * x * e2 + a[16] * 3.0f * z * (xx - yy) - a[17] * x * (xx + 3.0f * yy - 6.0f * zz)
          - a[18] * z * (3.0f * xx + 9.0f * yy - 4.0f * zz) + a[19] * 12.0f * y * e3
          - a[20] * 6.0f * xyz + a[21] * 4.0f * y * (yy - 3.0f * zz) - a[22] * 6.0f * xyz
          - a[23] * 4.0f * y * e1;
    gz += a[16] * y * e1 + a[17] * 12.0f * xyz - a[18] * 3.0f * y * e3
          - a[19] * 16.0f * z * (3.0f * xx + 3.0f * yy - 2.0f * zz) - a[20] * 3.0f * x * e3
          + a[21] * 12.0f * z * (xx - yy) + a[22] * x * e2;
}

// 4-body term from the l = 2 block s[0..4] = (xy, yz, 2zz-xx-yy, xz, xx-yy)
// sums: A = sum_j g (u u^T - I/3) is traceless symmetric with
// A_xy = s0, A_yz = s1, A_zz = s2/3, A_xz = s3, A_xx - A_yy = s4.
// q4 = tr(A^3); dq4/ds returned in ds.
template <class R>
NEP_HD R fourbody(const R* s, R* ds) {
    R axy = s[0], ayz = s[1], azz = s[2] * (R(1.0) / R(3.0)), axz = s[3];
    R axx = R(0.5) * (s[4] - azz), ayy = -R(0.5) * (s[4] + azz);
    // B = A^2 (symmetric)
    R bxx = axx * axx + axy * axy + axz * axz;
    R byy = axy * axy + ayy * ayy + ayz * ayz;
    R bzz = axz * axz + ayz * ayz + azz * azz;
    R bxy = axx * axy + axy * ayy + axz * ayz;
    R bxz = axx * axz + axy * ayz + axz * azz;
    R byz = axy * axz + ayy * ayz + ayz * azz;
    R q4 = axx * bxx + ayy * byy + azz * bzz + R(2.0) * (axy * bxy + axz * bxz + ayz * byz);
    if (ds) {
        ds[0] = R(6.0) * bxy;
        ds[1] = R(6.0) * byz;
        ds[2] = bzz - R(0.5) * (bxx + byy);
        ds[3] = R(6.0) * bxz;
        ds[4] = R(1.5) * (bxx - byy);
    }
    return q4;
}

NEP_HD float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
NEP_HD double fma_r(double a, double b, double c) { return fma(a, b, c); }

// Directional derivative of the 4-body gradient: J = dq4/ds (as fourbody)
// and dJ = d/de J(s + e ds) at e = 0.  With A(s) linear, d(A^2) = A dA + dA A
// and J is the same linear map of A^2 as dJ is of A dA + dA A.
template <class R>
NEP_HD void fourbody_jvp(const R* s, const R* ds, R* J, R* dJ) {
    R a[3][3], d[3][3];
    {
        const R azz = s[2] * (R(1.0) / R(3.0));
        a[0][1] = a[1][0] = s[0];
        a[1][2] = a[2][1] = s[1];
        a[0][2] = a[2][0] = s[3];
        a[2][2] = azz;
        a[0][0] = R(0.5) * (s[4] - azz);
        a[1][1] = -R(0.5) * (s[4] + azz);
        const R dzz = ds[2] * (R(1.0) / R(3.0));
        d[0][1] = d[1][0] = ds[0];
        d[1][2] = d[2][1] = ds[1];
        d[0][2] = d[2][0] = ds[3];
        d[2][2] = dzz;
        d[0][0] = R(0.5) * (ds[4] - dzz);
        d[1][1] = -R(0.5) * (ds[4] + dzz);
    }
    R B[3][3], C[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            R b = R(0.0), x = R(0.0), y = R(0.0);
            for (int k = 0; k < 3; ++k) {
                b = fma_r(a[r][k], a[k][c], b);
                x = fma_r(a[r][k], d[k][c], x);
                y = fma_r(d[r][k], a[k][c], y);
            }
            B[r][c] = b;
            C[r][c] = x + y;
        }
    J[0] = R(6.0) * B[0][1];
    J[1] = R(6.0) * B[1][2];
    J[2] = B[2][2] - R(0.5) * (B[0][0] + B[1][1]);
    J[3] = R(6.0) * B[0][2];
    J[4] = R(1.5) * (B[0][0] - B[1][1]);
    dJ[0] = R(6.0) * C[0][1];
    dJ[1] = R(6.0) * C[1][2];
    dJ[2] = C[2][2] - R(0.5) * (C[0][0] + C[1][1]);
    dJ[3] = R(6.0) * C[0][2];
    dJ[4] = R(1.5) * (C[0][0] - C[1][1]);
}

}  // namespace nep
