// lbpc_kernels.cuh -- device code of the coupled flow + enthalpy lattice Boltzmann step.
//
// Included once per storage precision by lbpc_kern_{f64,f32,f16,bf16}.cu, which define
// LBPC_PREC and the name of the launcher table.  Everything here is written for the
// structure of the two lattices (Eq. 3, Eq. 48) rather than with dense matrices: the
// D3Q19 moment transform (Eq. 51) is evaluated as grouped sums over the axis pairs and
// the three diagonal planes, and the D3Q7 MRT collision (Eq. 21-25) acts directly on
// the deviations g_a - g_a^eq of the six moving populations.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <cmath>
#include <cstring>

#include "lbpc_internal.h"

#define LBPC_HD __host__ __device__ __forceinline__

namespace lbpc {

// ---------------------------------------------------------------------------------
// Storage codecs.  Kernels compute on the stored representation r of a population: the
// value itself for FP64/FP32, its deviation from a fixed shift (the rest weight of f,
// (omega_T / 2) Cp_ref T_ref for g) for the 16-bit modes; the shift constants are folded
// into the arithmetic (Coef::frho, fm1, fm2, gshift).  16-bit values are also snapped to
// multiples of 2^-20 before rounding, so that a sum of six of them (each below 2 in
// magnitude) is exact in FP32: the enthalpy channel then needs no compensated sums.
// Only g needs the grid (enc_g); f is rounded plainly (enc).
// ---------------------------------------------------------------------------------
template <int P> struct Store;
template <> struct Store<LBPC_FP64> {
    using T = double; using C = double;
    static constexpr bool kGrid = false;
    static LBPC_HD C dec(T v, C) { return v; }
    static LBPC_HD T enc(C v, C) { return v; }
    static LBPC_HD T enc_g(C v, C) { return v; }
    static LBPC_HD C grid(C v) { return v; }
};
template <> struct Store<LBPC_FP32> {
    using T = float; using C = float;
    static constexpr bool kGrid = false;
    static LBPC_HD C dec(T v, C) { return v; }
    static LBPC_HD T enc(C v, C) { return v; }
    static LBPC_HD T enc_g(C v, C) { return v; }
    static LBPC_HD C grid(C v) { return v; }
};
// (v + 12) - 12 rounds v to a multiple of ulp(12) = 2^-20 for |v| < 4.
LBPC_HD float snap20(float v) { return (v + 12.0f) - 12.0f; }
template <> struct Store<LBPC_FP16S> {
    using T = __half; using C = float;
    static constexpr bool kGrid = true;
    static LBPC_HD C dec(T v, C) { return __half2float(v); }
    static LBPC_HD T enc(C v, C) { return __float2half_rn(v); }
    static LBPC_HD T enc_g(C v, C) { return __float2half_rn(snap20(v)); }
    static LBPC_HD C grid(C v) { return snap20(v); }
};
template <> struct Store<LBPC_BF16S> {
    using T = __nv_bfloat16; using C = float;
    static constexpr bool kGrid = true;
    static LBPC_HD C dec(T v, C) { return __bfloat162float(v); }
    static LBPC_HD T enc(C v, C) { return __float2bfloat16_rn(v); }
    static LBPC_HD T enc_g(C v, C) { return __float2bfloat16_rn(snap20(v)); }
    static LBPC_HD C grid(C v) { return snap20(v); }
};

// A storage mode fixes the precision of f (F) and of g (G): the four uniform modes, and
// 16-bit f with FP32 g, which keeps the enthalpy populations (and the wall fluxes they
// carry) at FP32 resolution for 140 instead of 116 bytes per node update.
template <int P> struct Mode { static constexpr int F = P, G = P; };
template <> struct Mode<LBPC_FP16S_G32> { static constexpr int F = LBPC_FP16S, G = LBPC_FP32; };
template <> struct Mode<LBPC_BF16S_G32> { static constexpr int F = LBPC_BF16S, G = LBPC_FP32; };
template <int P> using TF = typename Store<Mode<P>::F>::T;
template <int P> using TG = typename Store<Mode<P>::G>::T;
template <int P> using CT = typename Store<Mode<P>::F>::C;
// 16-bit f: the flow collision rebuilds f* from its moments (collide_flow)
template <int P> constexpr bool kRebuild = sizeof(TF<P>) == 2;

// Exact float -> double by integer operations (subnormal floats, below 1.2e-38, become
// zero); keeps the conversions off the FP64 pipe, which on GB300 issues a few
// operations per clock per SM.  Float infinities and NaN map to finite doubles, so a
// non-finite population does not reach the FP64 rest channel: divergence checks look at
// the populations themselves (macro_node, k_check).
LBPC_HD double f2d_exact(float v) {
#if defined(__CUDA_ARCH__)
    const unsigned u = __float_as_uint(v);
    const unsigned mag = u & 0x7fffffffu;
    const unsigned long long bits =
        mag < 0x00800000u ? 0ull
                          : ((unsigned long long)mag << 29) + (896ull << 52);
    return __longlong_as_double((long long)(bits | ((unsigned long long)(u >> 31) << 63)));
#else
    return (float)v == 0.0f || std::fabs(v) < 1.17549435e-38f ? 0.0 : (double)v;
#endif
}
// double -> float rounded to nearest (ties away from zero) by integer operations, off the
// FP64 pipe: the magnitude is truncated to the float's 23 mantissa bits and the first
// dropped bit is added (a carry into the exponent is the correct rounding).  Results below
// 2^-126 become signed zero (or the smallest subnormal); the inputs are finite enthalpy
// excesses.  (A ties-to-even version with a 64-bit rounding add, and the hardware
// conversion, both measured slower in the 16-bit step kernel.)
#if defined(__CUDA_ARCH__)
__device__ __forceinline__ float d2f_trunc(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((u >> 52) & 0x7ff) - 896;  // float biased exponent
    const unsigned sign = (unsigned)(u >> 63) << 31;
    if (ex <= 0) return __uint_as_float(sign);
    if (ex >= 255) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)ex << 23) | (unsigned)((u >> 29) & 0x7fffffu));
}
#endif
LBPC_HD float d2f_near(double v) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(__float_as_uint(d2f_trunc(v)) +
                           ((unsigned)(__double_as_longlong(v) >> 28) & 1u));
#else
    if (std::fabs(v) < 1.1754943508222875e-38) return std::signbit(v) ? -0.0f : 0.0f;
    return (float)v;
#endif
}

// Pairs of consecutive nodes along x: vector types and codecs of two values.
template <class T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<__half> { using type = __half2; };
template <> struct Vec2<__nv_bfloat16> { using type = __nv_bfloat162; };

template <int P> struct Pair;
template <> struct Pair<LBPC_FP64> {
    static LBPC_HD void dec(double2 v, double, double& a, double& b) { a = v.x; b = v.y; }
    static LBPC_HD double2 enc(double a, double b, double) { return make_double2(a, b); }
    static LBPC_HD double2 enc_g(double a, double b, double) { return make_double2(a, b); }
};
template <> struct Pair<LBPC_FP32> {
    static LBPC_HD void dec(float2 v, float, float& a, float& b) { a = v.x; b = v.y; }
    static LBPC_HD float2 enc(float a, float b, float) { return make_float2(a, b); }
    static LBPC_HD float2 enc_g(float a, float b, float) { return make_float2(a, b); }
};
template <> struct Pair<LBPC_FP16S> {
    static LBPC_HD void dec(__half2 v, float, float& a, float& b) {
        const float2 t = __half22float2(v);
        a = t.x;
        b = t.y;
    }
    static LBPC_HD __half2 enc(float a, float b, float) { return __floats2half2_rn(a, b); }
    static LBPC_HD __half2 enc_g(float a, float b, float) {
        return __floats2half2_rn(snap20(a), snap20(b));
    }
};
template <> struct Pair<LBPC_BF16S> {
    static LBPC_HD void dec(__nv_bfloat162 v, float, float& a, float& b) {
        const float2 t = __bfloat1622float2(v);
        a = t.x;
        b = t.y;
    }
    static LBPC_HD __nv_bfloat162 enc(float a, float b, float) {
        return __floats2bfloat162_rn(a, b);
    }
    static LBPC_HD __nv_bfloat162 enc_g(float a, float b, float) {
        return __floats2bfloat162_rn(snap20(a), snap20(b));
    }
};

template <class C> LBPC_HD const Coef<C>& coef(const Args& a);
template <> LBPC_HD const Coef<float>& coef<float>(const Args& a) { return a.cf; }
template <> LBPC_HD const Coef<double>& coef<double>(const Args& a) { return a.cd; }

// D3Q19 velocities in the order of Eq. 48: X(index, ex, ey, ez, opposite).
#define LBPC_Q19(X)                                                                     \
    X(0, 0, 0, 0, 0) X(1, 1, 0, 0, 2) X(2, -1, 0, 0, 1) X(3, 0, 1, 0, 4)                \
    X(4, 0, -1, 0, 3) X(5, 0, 0, 1, 6) X(6, 0, 0, -1, 5) X(7, 1, 1, 0, 10)              \
    X(8, -1, 1, 0, 9) X(9, 1, -1, 0, 8) X(10, -1, -1, 0, 7) X(11, 1, 0, 1, 14)          \
    X(12, -1, 0, 1, 13) X(13, 1, 0, -1, 12) X(14, -1, 0, -1, 11) X(15, 0, 1, 1, 18)     \
    X(16, 0, -1, 1, 17) X(17, 0, 1, -1, 16) X(18, 0, -1, -1, 15)
// D3Q7 moving velocities in the order of Eq. 3: X(index, ex, ey, ez, opposite).
#define LBPC_Q7(X)                                                                      \
    X(1, 1, 0, 0, 2) X(2, -1, 0, 0, 1) X(3, 0, 1, 0, 4) X(4, 0, -1, 0, 3)               \
    X(5, 0, 0, 1, 6) X(6, 0, 0, -1, 5)

// Neighbour access policies.  Nb: offsets (in nodes) to the neighbours at x-1 / x+1
// etc. with periodic wrap, and whether that neighbour lies behind a wall.  NbInterior:
// a node at least one cell away from every face, where every neighbour is a plain
// constant offset and no wall rule applies.
struct Nb {
    int oxm, oxp, oym, oyp, ozm, ozp;
    bool wxm, wxp, wym, wyp, wzm, wzp;
    // upwind neighbour x - e of velocity e = (EX, EY, EZ): offset and wall test
    template <int EX, int EY, int EZ>
    LBPC_HD int off() const {
        return (EX == 1 ? oxm : EX == -1 ? oxp : 0) + (EY == 1 ? oym : EY == -1 ? oyp : 0) +
               (EZ == 1 ? ozm : EZ == -1 ? ozp : 0);
    }
    template <int EX, int EY, int EZ>
    LBPC_HD bool wall() const {
        return (EX == 1 && wxm) || (EX == -1 && wxp) || (EY == 1 && wym) || (EY == -1 && wyp) ||
               (EZ == 1 && wzm) || (EZ == -1 && wzp);
    }
};

struct NbInterior {
    int sy, sz;  // node strides of y and z
    template <int EX, int EY, int EZ>
    LBPC_HD int off() const { return -EX - EY * sy - EZ * sz; }
    template <int EX, int EY, int EZ>
    LBPC_HD constexpr bool wall() const { return false; }
};

LBPC_HD Nb make_nb(const Args& a, int x, int y, int z) {
    Nb b;
    const int sy = a.nx, sz = a.nx * a.ny;
    b.oxm = (x == 0) ? a.nx - 1 : -1;
    b.oxp = (x == a.nx - 1) ? -(a.nx - 1) : 1;
    b.oym = (y == 0) ? (a.ny - 1) * sy : -sy;
    b.oyp = (y == a.ny - 1) ? -(a.ny - 1) * sy : sy;
    b.ozm = (z == 0) ? (a.nz - 1) * sz : -sz;
    b.ozp = (z == a.nz - 1) ? -(a.nz - 1) * sz : sz;
    b.wxm = (x == 0) && a.wall[0];
    b.wxp = (x == a.nx - 1) && a.wall[1];
    b.wym = (y == 0) && a.wall[2];
    b.wyp = (y == a.ny - 1) && a.wall[3];
    b.wzm = (z == 0) && a.wall[4];
    b.wzp = (z == a.nz - 1) && a.wall[5];
    return b;
}

LBPC_HD bool is_interior(const Args& a, int x, int y, int z) {
    return x > 0 && x < a.nx - 1 && y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1;
}

// Index of a node inside the temperature field of face `face`.
LBPC_HD int face_index(const Args& a, int face, int x, int y, int z) {
    return face < 2 ? y + a.ny * z : (face < 4 ? x + a.nx * z : x + a.nx * y);
}

template <class C>
LBPC_HD C fshift(const Coef<C>& k, int q) {
    return q == 0 ? k.fshift0 : (q < 7 ? k.fshift1 : k.fshift2);
}

// Anti-bounce-back source of a g population entering through face `face` (isothermal),
// in the representation: g_in = -g*_out + omega_T Cp_ref T_w, i.e. r_in = -r_out + this.
template <class C>
LBPC_HD C abb_source(const Args& a, const Coef<C>& k, int face, int x, int y, int z) {
    return k.wT_cref * (C)a.Tw[face][face_index(a, face, x, y, z)] - C(2) * k.gshift;
}

// ---------------------------------------------------------------------------------
// Gathers: pre-collision populations of node n for each memory layout.
// ---------------------------------------------------------------------------------
// 16-bit populations (and pairs of them): read-only loads that ask L2 to fetch 256 bytes
// around each miss; other types: plain read-only loads.
template <class X> struct Is16 { static constexpr bool value = false; };
template <> struct Is16<__half> { static constexpr bool value = true; };
template <> struct Is16<__nv_bfloat16> { static constexpr bool value = true; };
template <> struct Is16<__half2> { static constexpr bool value = true; };
template <> struct Is16<__nv_bfloat162> { static constexpr bool value = true; };
#if defined(__CUDA_ARCH__)
template <class X>
__device__ __forceinline__ X ld_nc(const X* p) {
    if constexpr (Is16<X>::value && sizeof(X) == 2) {
        unsigned short v;
        asm("ld.global.nc.L2::256B.u16 %0, [%1];" : "=h"(v) : "l"(p));
        return *reinterpret_cast<X*>(&v);
    } else if constexpr (Is16<X>::value && sizeof(X) == 4) {
        unsigned v;
        asm("ld.global.nc.L2::256B.u32 %0, [%1];" : "=r"(v) : "l"(p));
        return *reinterpret_cast<X*>(&v);
    } else {
        return __ldg(p);
    }
}
#endif
template <int P, int LAYOUT, bool NC>
LBPC_HD typename Store<P>::T ldv(const typename Store<P>::T* p) {
#if defined(__CUDA_ARCH__)
    if constexpr (NC) return ld_nc(p);
#endif
    return *p;
}

// Load of any type through the read-only path (device, NC) or plainly.
template <bool NC, class X>
LBPC_HD X ld_any(const X* p) {
#if defined(__CUDA_ARCH__)
    if constexpr (NC) return ld_nc(p);
#endif
    return *p;
}

template <int P, int LAYOUT, bool NC, class NB>
LBPC_HD void gather_f(const Args& a, const NB& b, int n,
                                         const typename Store<P>::T* fs,
                                         typename Store<P>::C* f) {
    using S = Store<P>;
    using C = typename S::C;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
#define LBPC_GF(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        int idx;                                                                        \
        int slot;                                                                       \
        if constexpr (LAYOUT == LAYOUT_AA_NATURAL) {                                    \
            idx = n; slot = q;                                                          \
        } else {                                                                        \
            const bool w = b.template wall<ex, ey, ez>();                                      \
            idx = w ? n : n + b.template off<ex, ey, ez>();                                    \
            if constexpr (LAYOUT == LAYOUT_PULL) slot = w ? op : q;                      \
            else slot = w ? q : op;                                                     \
        }                                                                               \
        f[q] = S::dec(ldv<P, LAYOUT, NC>(fs + (size_t)slot * N + idx), fshift(k, q));    \
    }
    LBPC_Q19(LBPC_GF)
#undef LBPC_GF
}

// g_1..6 (g[0] is not gathered: the rest population is the FP64 channel h').  The g
// lattice holds six planes: population q lives in plane q - 1.
template <int P, int LAYOUT, bool NC, class NB>
LBPC_HD void gather_g(const Args& a, const NB& b, int n, int x, int y, int z,
                                         const typename Store<P>::T* gs,
                                         typename Store<P>::C* g) {
    using S = Store<P>;
    using C = typename S::C;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
#define LBPC_GG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        if constexpr (LAYOUT == LAYOUT_AA_NATURAL) {                                    \
            g[q] = S::dec(ldv<P, LAYOUT, NC>(gs + (size_t)(q - 1) * N + n), k.gshift);         \
        } else {                                                                        \
            const bool w = b.template wall<ex, ey, ez>();                                      \
            const int idx = w ? n : n + b.template off<ex, ey, ez>();                          \
            int slot;                                                                   \
            if constexpr (LAYOUT == LAYOUT_PULL) slot = w ? op : q;                      \
            else slot = w ? q : op;                                                     \
            C v = S::dec(ldv<P, LAYOUT, NC>(gs + (size_t)(slot - 1) * N + idx), k.gshift);     \
            if (w && a.wall_iso[q - 1]) v = S::grid(-v + abb_source(a, k, q - 1, x, y, z)); \
            g[q] = v;                                                                   \
        }                                                                               \
    }
    LBPC_Q7(LBPC_GG)
#undef LBPC_GG
}

// ---------------------------------------------------------------------------------
// Scatters of post-collision populations.
// ---------------------------------------------------------------------------------
template <int P, int KIND, class NB>
LBPC_HD void scatter_f(const Args& a, const NB& b, int n,
                                          typename Store<P>::T* fd,
                                          const typename Store<P>::C* f) {
    using S = Store<P>;
    using C = typename S::C;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
#define LBPC_SF(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        const auto v = S::enc(f[q], fshift(k, q));                                      \
        if constexpr (KIND == STEP_PULL) {                                              \
            fd[(size_t)q * N + n] = v;                                                  \
        } else if constexpr (KIND == STEP_AA_EVEN) {                                    \
            fd[(size_t)op * N + n] = v;                                                 \
        } else { /* downwind neighbour x + e is the upwind neighbour of -e */           \
            const bool w = b.template wall<-(ex), -(ey), -(ez)>();                             \
            if (w) fd[(size_t)op * N + n] = v;                                          \
            else fd[(size_t)q * N + n + b.template off<-(ex), -(ey), -(ez)>()] = v;            \
        }                                                                               \
    }
    LBPC_Q19(LBPC_SF)
#undef LBPC_SF
}

// Stores g*_1..6 and replaces g[a] by the value as stored (rounded to the storage
// precision), which is what the downwind neighbours will read.
template <int P, int KIND, class NB>
LBPC_HD void scatter_g(const Args& a, const NB& b, int n, int x, int y, int z,
                       typename Store<P>::T* gd, typename Store<P>::C* g) {
    using S = Store<P>;
    using C = typename S::C;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
#define LBPC_SG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        const auto v = S::enc_g(g[q], k.gshift);                                        \
        g[q] = S::dec(v, k.gshift);                                                     \
        if constexpr (KIND == STEP_PULL) {                                              \
            gd[(size_t)(q - 1) * N + n] = v;                                                  \
        } else if constexpr (KIND == STEP_AA_EVEN) {                                    \
            gd[(size_t)(op - 1) * N + n] = v;                                                 \
        } else {                                                                        \
            const bool w = b.template wall<-(ex), -(ey), -(ez)>();                             \
            if (w) {                                                                    \
                auto vb = v;                                                            \
                if (a.wall_iso[op - 1])                                                 \
                    vb = S::enc_g(-S::dec(v, k.gshift) + abb_source(a, k, op - 1, x, y, z), \
                                  k.gshift);                                            \
                gd[(size_t)(op - 1) * N + n] = vb;                                            \
            } else {                                                                    \
                gd[(size_t)(q - 1) * N + n + b.template off<-(ex), -(ey), -(ez)>()] = v;             \
            }                                                                           \
        }                                                                               \
    }
    LBPC_Q7(LBPC_SG)
#undef LBPC_SG
}

// ---------------------------------------------------------------------------------
// Local physics.
// ---------------------------------------------------------------------------------

// Eq. 2 inverted (h = C_p T + f_l L; solid for h <= h_s, liquid for h >= h_s + L, mushy
// at T_m in between) from the FP64 enthalpy excess e = h - h_s that the rest channel
// carries, so that the cancelling subtraction near the melting point is exact.  FP64
// storage inverts in FP64, and so do the reported fields and diagnostics in every mode.
// The FP32 collision of the 32/16-bit modes inverts d = e rounded once to nearest (by
// integer operations, off the FP64 pipe): branch and value within half an FP32 ulp of e
// of the FP64 inversion; the branch can differ from the exact one only for e within half
// an ulp of 0 or L, where both branches give the same T and f_l to that accuracy.  (Exact
// branch tests on the bits of e measured 2% slower on the 16-bit step, an FP64 fused
// multiply-add for the value 5%.)
LBPC_HD void invert_excess(const Args& a, double e, double& T, double& fl) {
    const Coef<double>& k = a.cd;
    if (e <= 0.0) {
        fl = 0.0;
        T = k.Tm + e * k.Cps_inv;
    } else if (e >= k.L) {
        fl = 1.0;
        T = k.Tm + (e - k.L) * k.Cpl_inv;
    } else {
        fl = e * k.L_inv;
        T = k.Tm;
    }
}
LBPC_HD void invert_excess(const Args& a, double e, float& T, float& fl) {
    const Coef<float>& k = a.cf;
    const float d = d2f_near(e);
    if (d <= 0.0f) {
        fl = 0.0f;
        T = k.Tm + d * k.Cps_inv;
    } else if (d >= k.L) {
        fl = 1.0f;
        T = k.Tm + (d - k.L) * k.Cpl_inv;
    } else {
        fl = fminf(d * k.L_inv, 1.0f);
        T = k.Tm;
    }
}

// The excess taped for the adjoint, in the compute precision: exactly the value the
// forward inversion used (e itself for FP64, e rounded to nearest otherwise), so that the
// reverse sweep takes the forward's branch.
LBPC_HD double tape_excess(const Args&, double e, double) { return e; }
LBPC_HD float tape_excess(const Args&, double e, float) { return d2f_near(e); }

// Velocity factor phi of the solid closure, u = phi u*, F_s = -2 (1 - phi) rho0 u*: the
// liquid fraction itself, or with the enthalpy-porosity drag D = A (1 - f_l)^2 / (f_l^3 +
// eps), F_s = -D rho0 u and u = u* + F_s / (2 rho0) give phi = 1 / (1 + D / 2).  dphi (if
// given) receives dphi / df_l.
template <class C>
LBPC_HD C darcy_phi(const Coef<C>& k, C fl, C* dphi = nullptr) {
    const C s = C(1) - fl, q = fl * fl * fl + k.darcy_eps;
    const C D = k.darcy_A * s * s / q;
    const C phi = C(1) / (C(1) + C(0.5) * D);
    if (dphi) {
        const C dD = k.darcy_A * (C(-2) * s * q - C(3) * fl * fl * s * s) / (q * q);
        *dphi = C(-0.5) * phi * phi * dD;
    }
    return phi;
}
template <class C>
LBPC_HD C solid_phi(const Coef<C>& k, C fl, C* dphi = nullptr) {
    if (k.darcy) return darcy_phi(k, fl, dphi);
    if (dphi) *dphi = C(1);
    return fl;
}

// Density, momentum, Boussinesq force (Eq. 55), solid-phase force -2 (1 - phi) u* and the
// velocity of Eq. 56 (rho_0 = 1): u = phi (j + F_b / 2), phi = solid_phi(f_l).
template <class C>
LBPC_HD void flow_macro(const C* f, const Coef<C>& k, C T, C fl, C& rho, C& jx,
                                           C& jy, C& jz, C& ux, C& uy, C& uz, C& Fx, C& Fy,
                                           C& Fz) {
    rho = ((f[0] + (f[1] + f[2])) + ((f[3] + f[4]) + (f[5] + f[6]))) +
          (((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14])) +
           ((f[15] + f[16]) + (f[17] + f[18]))) + k.frho;
    jx = (f[1] - f[2]) + (f[7] - f[8] + f[9] - f[10]) + (f[11] - f[12] + f[13] - f[14]);
    jy = (f[3] - f[4]) + (f[7] + f[8] - f[9] - f[10]) + (f[15] - f[16] + f[17] - f[18]);
    jz = (f[5] - f[6]) + (f[11] + f[12] - f[13] - f[14]) + (f[15] + f[16] - f[17] - f[18]);
    const C Fb = k.gbeta * (T - k.Tref);
    const C usx = jx, usy = jy, usz = jz + C(0.5) * Fb;
    const C phi = solid_phi(k, fl);
    const C damp = C(-2) * (C(1) - phi);
    Fx = damp * usx;
    Fy = damp * usy;
    Fz = Fb + damp * usz;
    ux = phi * usx;
    uy = phi * usy;
    uz = phi * usz;
}

// Back-transform output: f*_a itself (RB) or the correction added to f_a.
template <bool RB, class C>
LBPC_HD void put_f(C& f, C v) {
    if constexpr (RB) f = v;
    else f += v;
}

// D3Q19 MRT collision with forcing (Eq. 49-54):
// f* = f + M^-1 [ -Lambda (m - m^eq) + (I - Lambda/2) FF ], with M^-1 = M^T diag(1/|row|^2).
// RB = false adds the correction to f.  RB = true rebuilds f* from its moments,
// f* = M^-1 [ m - Lambda (m - m^eq) + (I - Lambda/2) FF ] (M^-1 M = I), so the 19 inputs
// are not held to the end: fewer live registers, which lets the 16-bit pair kernels run
// six blocks per SM (FP32 keeps the correction form, which measured faster there).
template <bool RB, class C>
LBPC_HD void collide_flow(C* f, const Coef<C>& k, C T, C fl, C& ux, C& uy, C& uz, C& rho_o,
                          C& jx_o, C& jy_o, C& jz_o) {
    // grouped sums: axis pairs and the xy, xz, yz diagonal quadruples
    const C a1 = f[1] + f[2], b1 = f[1] - f[2];
    const C a3 = f[3] + f[4], b3 = f[3] - f[4];
    const C a5 = f[5] + f[6], b5 = f[5] - f[6];
    const C sxy = (f[7] + f[8]) + (f[9] + f[10]);
    const C xy_x = (f[7] - f[8]) + (f[9] - f[10]);
    const C xy_y = (f[7] + f[8]) - (f[9] + f[10]);
    const C xy_p = (f[7] - f[8]) - (f[9] - f[10]);
    const C sxz = (f[11] + f[12]) + (f[13] + f[14]);
    const C xz_x = (f[11] - f[12]) + (f[13] - f[14]);
    const C xz_z = (f[11] + f[12]) - (f[13] + f[14]);
    const C xz_p = (f[11] - f[12]) - (f[13] - f[14]);
    const C syz = (f[15] + f[16]) + (f[17] + f[18]);
    const C yz_y = (f[15] - f[16]) + (f[17] - f[18]);
    const C yz_z = (f[15] + f[16]) - (f[17] + f[18]);
    const C yz_p = (f[15] - f[16]) - (f[17] - f[18]);
    const C sax = a1 + a3 + a5, sdg = sxy + sxz + syz;

    const C rst = f[0] + sax + sdg;  // rho of the stored representation
    const C rho = rst + k.frho;
    const C tx = xy_x + xz_x, ty = xy_y + yz_y, tz = xz_z + yz_z;
    const C jx = b1 + tx, jy = b3 + ty, jz = b5 + tz;
    rho_o = rho;
    jx_o = jx;
    jy_o = jy;
    jz_o = jz;
    // non-conserved moments (rows 4, 6, 8-18 of Eq. 51); rows 1 and 2 enter below only as
    // m1 - m1eq = 19 (sdg - f0 - rho u^2) and m2 - m2eq = 9 f0 - 7 sax - 2 sdg + 5.5 rho u^2,
    // where the rest-weight constants of the stored representation cancel
    const C m4 = tx - C(4) * b1, m6 = ty - C(4) * b3, m8 = tz - C(4) * b5;
    const C a35 = a3 + a5, h9 = (sxy + sxz) - C(2) * syz;
    const C m9 = C(2) * a1 - a35 + h9;
    const C m10 = C(2) * a35 - C(4) * a1 + h9;
    const C k11 = sxy - sxz, a53 = a5 - a3;
    const C m11 = k11 - a53, m12 = C(2) * a53 + k11;
    const C m16 = xy_x - xz_x, m17 = yz_y - xy_y, m18 = xz_z - yz_z;

    // forces and velocity (Eq. 55-56 with the solid-phase force)
    const C Fb = k.gbeta * (T - k.Tref);
    const C usx = jx, usy = jy, usz = jz + C(0.5) * Fb;
    const C damp = C(-2) * (C(1) - fl);
    const C Fx = damp * usx, Fy = damp * usy, Fz = Fb + damp * usz;
    ux = fl * usx;
    uy = fl * usy;
    uz = fl * usz;

    // equilibrium moments (Eq. 53) and forcing moments (Eq. 54), c = 1
    const C uxx = ux * ux, uyy = uy * uy, uzz = uz * uz, u2 = uxx + uyy + uzz;
    const C Fu = Fx * ux + Fy * uy + Fz * uz;
    const C ru2 = rho * u2, rux = rho * ux;
    const C pxx_eq = rho * (C(3) * uxx - u2), pww_eq = rho * (uyy - uzz);
    const C FFxx = C(6) * Fx * ux - C(2) * Fu, FFww = C(2) * (Fy * uy - Fz * uz);

    // d_k = [-s_k (m_k - meq_k) + (1 - s_k/2) FF_k] / |row k|^2 (correction form), or with RB
    // m*_k / |row k|^2 = d_k + m_k / |row k|^2 = [(1 - s_k) m_k + s_k meq_k + (1 - s_k/2)
    // FF_k] / |row k|^2; the products of the rates, (1 - s_k/2), (1 - s_k) and 1/|row k|^2
    // are folded into the r_*, c_* and k_* constants on the host.  With RB, rows 0-2 leave
    // out the rest-weight moments (1, -11, 3) rho_st of the stored representation, which
    // enter the back-transform as w_a rho_st
    C d1, d2, d3, d4, d5, d6, d7, d8, d9, d10, d11, d12, d13, d14, d15, d16, d17, d18;
    if constexpr (RB) {
        const C rq23 = k.r_q * (C(2.0 / 3.0) * rho);
        d1 = k.k_e * (sdg - f[0]) - k.r_e * ru2 + k.c_e * Fu;
        d2 = k.k_eps * (C(9) * f[0] - C(7) * sax - C(2) * sdg) + C(5.5) * k.r_eps * ru2 +
             k.c_eps * Fu;
        d3 = (jx + Fx) * C(0.1), d5 = (jy + Fy) * C(0.1), d7 = (jz + Fz) * C(0.1);
        d4 = k.k_q * m4 + rq23 * ux + k.c_q * Fx;
        d6 = k.k_q * m6 + rq23 * uy + k.c_q * Fy;
        d8 = k.k_q * m8 + rq23 * uz + k.c_q * Fz;
        d9 = k.k_nu9 * m9 - k.r_nu9 * pxx_eq + k.c_nu9 * FFxx;
        d10 = k.k_pi10 * m10 + C(0.5) * k.r_pi10 * pxx_eq + k.c_pi10 * FFxx;
        d11 = k.k_nu11 * m11 - k.r_nu11 * pww_eq + k.c_nu11 * FFww;
        d12 = k.k_pi12 * m12 + C(0.5) * k.r_pi12 * pww_eq + k.c_pi12 * FFww;
        d13 = k.k_nu13 * xy_p - k.r_nu13 * (rux * uy) + k.c_nu13 * (Fx * uy + Fy * ux);
        d14 = k.k_nu13 * yz_p - k.r_nu13 * (rho * uy * uz) + k.c_nu13 * (Fy * uz + Fz * uy);
        d15 = k.k_nu13 * xz_p - k.r_nu13 * (rux * uz) + k.c_nu13 * (Fx * uz + Fz * ux);
        d16 = k.k_t * m16, d17 = k.k_t * m17, d18 = k.k_t * m18;
    } else {
        const C r23 = C(2.0 / 3.0) * rho;
        d1 = k.r_e * (sdg - f[0] - ru2) + k.c_e * Fu;
        d2 = k.r_eps * (C(9) * f[0] - C(7) * sax - C(2) * sdg + C(5.5) * ru2) + k.c_eps * Fu;
        d3 = Fx * C(0.1), d5 = Fy * C(0.1), d7 = Fz * C(0.1);
        d4 = k.r_q * (m4 + r23 * ux) + k.c_q * Fx;
        d6 = k.r_q * (m6 + r23 * uy) + k.c_q * Fy;
        d8 = k.r_q * (m8 + r23 * uz) + k.c_q * Fz;
        d9 = k.r_nu9 * (m9 - pxx_eq) + k.c_nu9 * FFxx;
        d10 = k.r_pi10 * (m10 + C(0.5) * pxx_eq) + k.c_pi10 * FFxx;
        d11 = k.r_nu11 * (m11 - pww_eq) + k.c_nu11 * FFww;
        d12 = k.r_pi12 * (m12 + C(0.5) * pww_eq) + k.c_pi12 * FFww;
        d13 = k.r_nu13 * (xy_p - rux * uy) + k.c_nu13 * (Fx * uy + Fy * ux);
        d14 = k.r_nu13 * (yz_p - rho * uy * uz) + k.c_nu13 * (Fy * uz + Fz * uy);
        d15 = k.r_nu13 * (xz_p - rux * uz) + k.c_nu13 * (Fx * uz + Fz * ux);
        d16 = k.r_t * m16, d17 = k.r_t * m17, d18 = k.r_t * m18;
    }

    // back-transform: sum_k M_ka d_k (columns of Eq. 51; with RB plus w_a rho_st, as M w =
    // (1, -11, 3, 0, ...)), with the sums shared between the members of each axis pair and
    // diagonal quadruple
    C e0, eax, edg;
    if constexpr (RB) {
        e0 = rst * C(1.0 / 3.0) + C(-30) * d1 + C(12) * d2;
        eax = rst * C(1.0 / 18.0) + C(-11) * d1 - C(4) * d2;
        edg = rst * C(1.0 / 36.0) + C(8) * d1 + d2;
    } else {
        e0 = C(-30) * d1 + C(12) * d2;
        eax = C(-11) * d1 - C(4) * d2;
        edg = C(8) * d1 + d2;
    }
    put_f<RB>(f[0], e0);
    const C ox = d3 - C(4) * d4, oy = d5 - C(4) * d6, oz = d7 - C(4) * d8;
    const C ex1 = eax + C(2) * d9 - C(4) * d10;
    const C cyz = eax - d9 + C(2) * d10, w11 = d11 - C(2) * d12;
    const C ey1 = cyz + w11, ez1 = cyz - w11;
    put_f<RB>(f[1], ex1 + ox);
    put_f<RB>(f[2], ex1 - ox);
    put_f<RB>(f[3], ey1 + oy);
    put_f<RB>(f[4], ey1 - oy);
    put_f<RB>(f[5], ez1 + oz);
    put_f<RB>(f[6], ez1 - oz);
    const C X = d3 + d4, Y = d5 + d6, Z = d7 + d8;
    const C a910 = edg + d9 + d10, b1112 = d11 + d12;
    const C exy = a910 + b1112, exz = a910 - b1112;
    const C eyz = edg - C(2) * d9 - C(2) * d10;
    {  // xy: f7..f10 = e_xy +-(d13) + (+-X +-Y) + (+-d16 -+d17)
        const C u = X + d16, v = Y - d17, P = exy + d13, Q = exy - d13;
        const C s = u + v, w = v - u;
        put_f<RB>(f[7], P + s);
        put_f<RB>(f[8], Q + w);
        put_f<RB>(f[9], Q - w);
        put_f<RB>(f[10], P - s);
    }
    {  // xz: f11..f14
        const C u = X - d16, v = Z + d18, P = exz + d15, Q = exz - d15;
        const C s = u + v, w = v - u;
        put_f<RB>(f[11], P + s);
        put_f<RB>(f[12], Q + w);
        put_f<RB>(f[13], Q - w);
        put_f<RB>(f[14], P - s);
    }
    {  // yz: f15..f18
        const C u = Y + d17, v = Z - d18, P = eyz + d14, Q = eyz - d14;
        const C s = u + v, w = v - u;
        put_f<RB>(f[15], P + s);
        put_f<RB>(f[16], Q + w);
        put_f<RB>(f[17], Q - w);
        put_f<RB>(f[18], P - s);
    }
}

// D3Q7 enthalpy collision on the six moving populations (Eq. 21-25; SRT when every
// rate equals 1/tau_g).  With d_a = g_a - g_a^eq, d_0 = -sum d_a (h is conserved), the
// moments of d are m1..m3 (odd pairs), m4 = -7 S, m5, m6; g* = g^eq + d - N^-1 R N d.
// VAR (conduction kernels): with per-phase conductivities the rates follow from f_l.
template <class C, bool VAR = false>
LBPC_HD void collide_enth(C* g, const Coef<C>& k, C T, C fl, C ux, C uy, C uz) {
    const C Cp = k.Cps + fl * k.dCp;
    // an axis pair's equilibria (Eq. 7) sum to cT2 (representation) and differ by vT2 u
    const C cT2 = k.wT_cref * T - k.gshift2;
    const C vT2 = Cp * T;
    // moments of d = g - g^eq: odd pair differences m1..m3, pair sums p
    const C m1 = (g[1] - g[2]) - vT2 * ux;
    const C m2 = (g[3] - g[4]) - vT2 * uy;
    const C m3 = (g[5] - g[6]) - vT2 * uz;
    const C p12 = (g[1] + g[2]) - cT2, p34 = (g[3] + g[4]) - cT2, p56 = (g[5] + g[6]) - cT2;
    const C q = p34 + p56;
    const C S = p12 + q, m5 = C(2) * p12 - q, m6 = p34 - p56;
    // g* = g^eq + d - N^-1 R N d = g - N^-1 R N d, rates and 1/|row|^2 folded on the host
    C s46 = k.sig4_6, s56 = k.sig5_6, s64 = k.sig6_4, hchi = k.hchi;
    if (VAR && k.varchi) {  // Eq. 34 per node, lambda(f_l) linear in f_l
        const C sc = C(1) / (k.chi_a + k.chi_b * fl);
        const C s4 = k.s4_a + k.s4_b * sc;
        s46 = s4 * C(1.0 / 6.0);
        s56 = s46;
        s64 = s4 * C(0.25);
        hchi = C(0.5) * sc;
    }
    const C A = s46 * S, B = s56 * m5, D = s64 * m6;
    const C c12 = A + B, c36 = A - C(0.5) * B;
    const C c3p = c36 + D, c3m = c36 - D;
    const C h1 = hchi * m1, h2 = hchi * m2, h3 = hchi * m3;
    g[1] -= c12 + h1;
    g[2] -= c12 - h1;
    g[3] -= c3p + h2;
    g[4] -= c3p - h2;
    g[5] -= c3m + h3;
    g[6] -= c3m - h3;
}

// The rest channel stores e' = h' - h_s in FP64, so that e = h - h_s = e' + sum_{a>=1} g_a.
// With 32/16-bit populations the six values are summed exactly in FP32 (Knuth's TwoSum:
// s + err == a + b) into an unevaluated pair hi + lo, and only the pair enters FP64:
// four FP64 additions and five conversions per node instead of a dozen of each.
LBPC_HD void two_sum(float a, float b, float& s, float& err) {
    s = a + b;
    const float bb = s - a;
    err = (a - (s - bb)) + (b - bb);
}
LBPC_HD void sum6_pair(const float* g, float& hi, float& lo) {
    float e;
    hi = g[1];
    lo = 0.0f;
    two_sum(hi, g[2], hi, e); lo += e;
    two_sum(hi, g[3], hi, e); lo += e;
    two_sum(hi, g[4], hi, e); lo += e;
    two_sum(hi, g[5], hi, e); lo += e;
    two_sum(hi, g[6], hi, e); lo += e;
}
// e' + sum g_a and e - sum g_a.  FP64: plain FP64 sums.  FP32 storage: exact FP32 pair
// sums (TwoSum).  16-bit storage: the six values lie on a 2^-20 grid, so a plain FP32
// sum is already exact.
template <int P>
LBPC_HD double excess_plus(double ep, const typename Store<P>::C* g) {
    if constexpr (P == LBPC_FP64) {
        return ep + g[1] + g[2] + g[3] + g[4] + g[5] + g[6];
    } else if constexpr (Store<P>::kGrid) {
        return ep + f2d_exact(((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]));
    } else {
        float hi, lo;
        sum6_pair(g, hi, lo);
        return (ep + f2d_exact(hi)) + f2d_exact(lo);
    }
}
template <int P>
LBPC_HD double excess_minus(double e, const typename Store<P>::C* g) {
    if constexpr (P == LBPC_FP64) {
        return e - g[1] - g[2] - g[3] - g[4] - g[5] - g[6];
    } else if constexpr (Store<P>::kGrid) {
        return e - f2d_exact(((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]));
    } else {
        float hi, lo;
        sum6_pair(g, hi, lo);
        return (e - f2d_exact(hi)) - f2d_exact(lo);
    }
}

// ---------------------------------------------------------------------------------
// Node-level operations (host + device: the kernels below call them once per node).
// ---------------------------------------------------------------------------------
constexpr int STEP_THREADS = 128;
// Largest lattice the pair paths take: they form plane offsets of up to 3 N in int.
constexpr int kPairMaxN = 715827882;  // floor((2^31 - 1) / 3)

template <int KIND> struct KindLayout;
template <> struct KindLayout<STEP_PULL> { static constexpr int value = LAYOUT_PULL; };
template <> struct KindLayout<STEP_AA_EVEN> { static constexpr int value = LAYOUT_AA_NATURAL; };
template <> struct KindLayout<STEP_AA_ODD> { static constexpr int value = LAYOUT_AA_SWAPPED; };

// One time step of node (x, y, z): gather (stream in, with wall rules), Eq. 2 inversion,
// flow collision, enthalpy collision, scatter, FP64 rest channel update.
template <int P, int KIND, int FLOW, bool TAPE = false>
LBPC_HD void step_node(const Args& a, int x, int y, int z, const TF<P>* fs,
                       TF<P>* fd, const TG<P>* gs,
                       TG<P>* gd, double* hp, CT<P>* tape_e = nullptr,
                       CT<P>* tape_m = nullptr) {
    using C = CT<P>;
    const Coef<C>& k = coef<C>(a);
    const int n = x + a.nx * (y + a.ny * z);
    constexpr int LAYOUT = KindLayout<KIND>::value;
    constexpr bool NC = KIND == STEP_PULL;  // read-only path only when src != dst
    const bool interior = is_interior(a, x, y, z);
    const NbInterior bi{a.nx, a.nx * a.ny};
    const Nb b = make_nb(a, x, y, z);

    C f[19], g[7];
    if (interior) {
        if constexpr (FLOW) gather_f<Mode<P>::F, LAYOUT, NC>(a, bi, n, fs, f);
        gather_g<Mode<P>::G, LAYOUT, NC>(a, bi, n, x, y, z, gs, g);
    } else {
        if constexpr (FLOW) gather_f<Mode<P>::F, LAYOUT, NC>(a, b, n, fs, f);
        gather_g<Mode<P>::G, LAYOUT, NC>(a, b, n, x, y, z, gs, g);
    }
    const double e = excess_plus<Mode<P>::G>(hp[n], g);  // h - h_s

    C T, fl;
    invert_excess(a, e, T, fl);
    C ux = C(0), uy = C(0), uz = C(0), rho = C(0), jx = C(0), jy = C(0), jz = C(0);
    if constexpr (FLOW)  // FLOW 2: the drag closure, phi(f_l) in place of f_l
        collide_flow<kRebuild<P>>(f, k, T, FLOW == 2 ? darcy_phi(k, fl) : fl, ux, uy, uz, rho, jx,
                                  jy, jz);
    if constexpr (TAPE) {  // macroscopic tape of the pre-collision state (adjoint)
        tape_e[n] = tape_excess(a, e, C(0));
        if constexpr (FLOW) {
            tape_m[n] = rho;
            tape_m[(size_t)a.N + n] = jx;
            tape_m[2 * (size_t)a.N + n] = jy;
            tape_m[3 * (size_t)a.N + n] = jz;
        }
    }
    collide_enth<C, !FLOW>(g, k, T, fl, ux, uy, uz);
    if (interior) {
        if constexpr (FLOW) scatter_f<Mode<P>::F, KIND>(a, bi, n, fd, f);
        scatter_g<Mode<P>::G, KIND>(a, bi, n, x, y, z, gd, g);
    } else {
        if constexpr (FLOW) scatter_f<Mode<P>::F, KIND>(a, b, n, fd, f);
        scatter_g<Mode<P>::G, KIND>(a, b, n, x, y, z, gd, g);
    }
    hp[n] = excess_minus<Mode<P>::G>(e, g);
}


// Inversion and both collisions of a node pair (n0, n0 + 1), in registers; with TAPE also
// the macroscopic tape of the pair's pre-collision state (adjoint).
template <int P, int FLOW, bool TAPE = false>
LBPC_HD void pair_collide(const Args& a, CT<P>* f0, CT<P>* f1, CT<P>* g0, CT<P>* g1, double e0,
                          double e1, int n0 = 0, CT<P>* tape_e = nullptr,
                          CT<P>* tape_m = nullptr) {
    using C = CT<P>;
    using VC = typename Vec2<C>::type;
    const Coef<C>& k = coef<C>(a);
    C T0, fl0, T1, fl1;
    invert_excess(a, e0, T0, fl0);
    invert_excess(a, e1, T1, fl1);
    C ux0 = C(0), uy0 = C(0), uz0 = C(0), ux1 = C(0), uy1 = C(0), uz1 = C(0);
    if constexpr (FLOW) {
        C r0, jx0, jy0, jz0, r1, jx1, jy1, jz1;
        collide_flow<kRebuild<P>>(f0, k, T0, FLOW == 2 ? darcy_phi(k, fl0) : fl0, ux0, uy0, uz0,
                                  r0, jx0, jy0, jz0);
        collide_flow<kRebuild<P>>(f1, k, T1, FLOW == 2 ? darcy_phi(k, fl1) : fl1, ux1, uy1, uz1,
                                  r1, jx1, jy1, jz1);
        if constexpr (TAPE) {
            const size_t N = (size_t)a.N;
            *reinterpret_cast<VC*>(tape_m + n0) = VC{r0, r1};
            *reinterpret_cast<VC*>(tape_m + N + n0) = VC{jx0, jx1};
            *reinterpret_cast<VC*>(tape_m + 2 * N + n0) = VC{jy0, jy1};
            *reinterpret_cast<VC*>(tape_m + 3 * N + n0) = VC{jz0, jz1};
        }
    }
    if constexpr (TAPE)
        *reinterpret_cast<VC*>(tape_e + n0) = VC{tape_excess(a, e0, C(0)), tape_excess(a, e1, C(0))};
    collide_enth<C, !FLOW>(g0, k, T0, fl0, ux0, uy0, uz0);
    collide_enth<C, !FLOW>(g1, k, T1, fl1, ux1, uy1, uz1);
}

// Two nodes (x0, x0 + 1), x0 even, of a row away from every y and z face: populations
// with e_x = 0 move as aligned pairs; e_x = +-1 ones are two scalar loads, with the x-face
// rules (periodic wrap; at a wall the reflected population of the node itself) applied
// by selecting a 32-bit element offset from the population's plane on the lanes at x = 0
// / x = nx - 1; every store is a pair.  Requires even nx.
template <int P, int FLOW, bool TAPE = false>
LBPC_HD void step_pair_pull(const Args& a, int x0, int y, int z, const TF<P>* fs,
                            TF<P>* fd, const TG<P>* gs,
                            TG<P>* gd, double* hp, CT<P>* tape_e = nullptr,
                            CT<P>* tape_m = nullptr) {
    using SF = Store<Mode<P>::F>;
    using SG = Store<Mode<P>::G>;
    using TFt = typename SF::T;
    using TGt = typename SG::T;
    using C = CT<P>;
    using VF = typename Vec2<TFt>::type;
    using VG = typename Vec2<TGt>::type;
    using PRF = Pair<Mode<P>::F>;
    using PRG = Pair<Mode<P>::G>;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
    const int N32 = a.N;  // 3 N < 2^31 (kPairMaxN)
    const int sy = a.nx, sz = a.nx * a.ny;
    const int n0 = x0 + a.nx * (y + a.ny * z), n1 = n0 + 1;
    const bool xlo = x0 == 0, xhi = x0 + 1 == a.nx - 1;
    const bool wlo = xlo && a.wall[0], whi = xhi && a.wall[1];
    // upwind x-neighbour of node 0 for e_x = +1 and of node 1 for e_x = -1 (with wrap)
    const int up0 = xlo ? n0 + a.nx - 1 : n0 - 1;
    const int up1 = xhi ? n1 - (a.nx - 1) : n1 + 1;
    C f0[19], f1[19], g0[7], g1[7];
    if constexpr (FLOW) {
#define LBPC_PF(q, ex, ey, ez, op)                                                       \
        {                                                                               \
            const int oyz = -(ey) * sy - (ez) * sz;                                     \
            const C sh = fshift(k, q);                                                  \
            const TFt* pl = fs + (size_t)q * N;                                           \
            if constexpr ((ex) == 0) {                                                  \
                PRF::dec(ld_any<true>(reinterpret_cast<const VF*>(pl + n0 + oyz)),             \
                        sh, f0[q], f1[q]);                                              \
            } else if constexpr ((ex) == 1) {                                           \
                const int i0 = wlo ? ((op) - (q)) * N32 + n0 : up0 + oyz;               \
                f0[q] = SF::dec(ldv<Mode<P>::F, LAYOUT_PULL, true>(pl + i0), sh);                 \
                f1[q] = SF::dec(ldv<Mode<P>::F, LAYOUT_PULL, true>(pl + n0 + oyz), sh);           \
            } else {                                                                    \
                const int i1 = whi ? ((op) - (q)) * N32 + n1 : up1 + oyz;               \
                f0[q] = SF::dec(ldv<Mode<P>::F, LAYOUT_PULL, true>(pl + n1 + oyz), sh);           \
                f1[q] = SF::dec(ldv<Mode<P>::F, LAYOUT_PULL, true>(pl + i1), sh);                 \
            }                                                                           \
        }
        LBPC_Q19(LBPC_PF)
#undef LBPC_PF
    }
#define LBPC_PG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        const int oyz = -(ey) * sy - (ez) * sz;                                         \
        const TGt* pl = gs + (size_t)(q - 1) * N;                                         \
        if constexpr ((ex) == 0) {                                                      \
            PRG::dec(ld_any<true>(reinterpret_cast<const VG*>(pl + n0 + oyz)),                 \
                    k.gshift, g0[q], g1[q]);                                            \
        } else if constexpr ((ex) == 1) {                                               \
            const int i0 = wlo ? ((op) - (q)) * N32 + n0 : up0 + oyz;                   \
            C v = SG::dec(ldv<Mode<P>::G, LAYOUT_PULL, true>(pl + i0), k.gshift);                 \
            if (wlo && a.wall_iso[0]) v = SG::grid(-v + abb_source(a, k, 0, x0, y, z)); \
            g0[q] = v;                                                                  \
            g1[q] = SG::dec(ldv<Mode<P>::G, LAYOUT_PULL, true>(pl + n0 + oyz), k.gshift);         \
        } else {                                                                        \
            const int i1 = whi ? ((op) - (q)) * N32 + n1 : up1 + oyz;                   \
            C v = SG::dec(ldv<Mode<P>::G, LAYOUT_PULL, true>(pl + i1), k.gshift);                 \
            if (whi && a.wall_iso[1]) v = SG::grid(-v + abb_source(a, k, 1, x0 + 1, y, z)); \
            g1[q] = v;                                                                  \
            g0[q] = SG::dec(ldv<Mode<P>::G, LAYOUT_PULL, true>(pl + n1 + oyz), k.gshift);         \
        }                                                                               \
    }
    LBPC_Q7(LBPC_PG)
#undef LBPC_PG
    const double2 ep = ld_any<true>(reinterpret_cast<const double2*>(hp + n0));
    const double e0 = excess_plus<Mode<P>::G>(ep.x, g0), e1 = excess_plus<Mode<P>::G>(ep.y, g1);
    pair_collide<P, FLOW, TAPE>(a, f0, f1, g0, g1, e0, e1, n0, tape_e, tape_m);
    if constexpr (FLOW) {
#define LBPC_SPF(q, ex, ey, ez, op)                                                      \
        *reinterpret_cast<VF*>(fd + (size_t)q * N + n0) = PRF::enc(f0[q], f1[q], fshift(k, q));
        LBPC_Q19(LBPC_SPF)
#undef LBPC_SPF
    }
#define LBPC_SPG(q, ex, ey, ez, op)                                                      \
    {                                                                                   \
        const VG v = PRG::enc_g(g0[q], g1[q], k.gshift);                                \
        *reinterpret_cast<VG*>(gd + (size_t)(q - 1) * N + n0) = v;                       \
        PRG::dec(v, k.gshift, g0[q], g1[q]);                                            \
    }
    LBPC_Q7(LBPC_SPG)
#undef LBPC_SPG
    *reinterpret_cast<double2*>(hp + n0) = make_double2(excess_minus<Mode<P>::G>(e0, g0), excess_minus<Mode<P>::G>(e1, g1));
}


// Hides v's value from the compiler: the scatter addresses of an AA step are gather
// addresses (the same slots, in place), and without this the compiler keeps them all live
// across the collision.
template <class T>
LBPC_HD void opaque(T& v) {
#if defined(__CUDA_ARCH__)
    if constexpr (sizeof(T) == 8) asm volatile("" : "+l"(v));
    else asm volatile("" : "+r"(v));
#else
    (void)v;
#endif
}

// AA in-place streaming, two nodes (x0, x0 + 1) per thread, row away from the y/z faces.
// Even step (natural layout): every access is a local aligned pair; f*_q goes to slot qbar.
// Odd step (swapped layout): f_q(x) is slot qbar at x - e_q (slot q at x behind a wall) and
// f*_q goes to slot q at x + e_q (slot qbar at x behind a wall), with the wall rules of the
// per-node path.  Each thread reads and writes the same set of slots, so in place is safe.
template <int P, int FLOW, bool ODD>
LBPC_HD void step_pair_aa(const Args& a, int x0, int y, int z, TF<P>* F, TG<P>* G, double* hp) {
    using SF = Store<Mode<P>::F>;
    using SG = Store<Mode<P>::G>;
    using TFt = typename SF::T;
    using TGt = typename SG::T;
    using C = CT<P>;
    using VF = typename Vec2<TFt>::type;
    using VG = typename Vec2<TGt>::type;
    using PRF = Pair<Mode<P>::F>;
    using PRG = Pair<Mode<P>::G>;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
    const int N32 = a.N;  // 3 N < 2^31 (kPairMaxN)
    const int sy = a.nx, sz = a.nx * a.ny;
    const int n0 = x0 + a.nx * (y + a.ny * z), n1 = n0 + 1;
    const bool xlo = x0 == 0, xhi = x0 + 1 == a.nx - 1;
    const bool wlo = xlo && a.wall[0], whi = xhi && a.wall[1];
    const int dn0 = xlo ? n0 + a.nx - 1 : n0 - 1;      // x-neighbour x0 - 1 (wrapped)
    const int up1 = xhi ? n1 - (a.nx - 1) : n1 + 1;    // x-neighbour x1 + 1 (wrapped)
    C f0[19], f1[19], g0[7], g1[7];
    // ---- gather ----
    if constexpr (FLOW) {
#define LBPC_AGF(q, ex, ey, ez, op)                                                      \
        {                                                                               \
            const C sh = fshift(k, q);                                                  \
            if constexpr (!ODD) {                                                       \
                PRF::dec(*reinterpret_cast<const VF*>(F + (size_t)q * N + n0), sh, f0[q], f1[q]); \
            } else {                                                                    \
                const int oyz = -(ey) * sy - (ez) * sz;                                 \
                const TFt* sw = F + (size_t)op * N;                                     \
                if constexpr ((ex) == 0) {                                              \
                    PRF::dec(*reinterpret_cast<const VF*>(sw + n0 + oyz), sh, f0[q], f1[q]); \
                } else if constexpr ((ex) == 1) {                                       \
                    f0[q] = SF::dec(sw[wlo ? ((q) - (op)) * N32 + n0 : dn0 + oyz], sh);  \
                    f1[q] = SF::dec(sw[n0 + oyz], sh);                                \
                } else {                                                                \
                    f0[q] = SF::dec(sw[n1 + oyz], sh);                                \
                    f1[q] = SF::dec(sw[whi ? ((q) - (op)) * N32 + n1 : up1 + oyz], sh);  \
                }                                                                       \
            }                                                                           \
        }
        LBPC_Q19(LBPC_AGF)
#undef LBPC_AGF
    }
#define LBPC_AGG(q, ex, ey, ez, op)                                                      \
    {                                                                                   \
        if constexpr (!ODD) {                                                           \
            PRG::dec(*reinterpret_cast<const VG*>(G + (size_t)(q - 1) * N + n0), k.gshift, g0[q], g1[q]); \
        } else {                                                                        \
            const int oyz = -(ey) * sy - (ez) * sz;                                     \
            const TGt* sw = G + (size_t)(op - 1) * N;                                   \
            if constexpr ((ex) == 0) {                                                  \
                PRG::dec(*reinterpret_cast<const VG*>(sw + n0 + oyz), k.gshift, g0[q], g1[q]); \
            } else if constexpr ((ex) == 1) {                                           \
                C v = SG::dec(sw[wlo ? ((q) - (op)) * N32 + n0 : dn0 + oyz], k.gshift);  \
                if (wlo && a.wall_iso[0]) v = SG::grid(-v + abb_source(a, k, 0, x0, y, z)); \
                g0[q] = v;                                                              \
                g1[q] = SG::dec(sw[n0 + oyz], k.gshift);                                    \
            } else {                                                                    \
                g0[q] = SG::dec(sw[n1 + oyz], k.gshift);                                    \
                C v = SG::dec(sw[whi ? ((q) - (op)) * N32 + n1 : up1 + oyz], k.gshift);  \
                if (whi && a.wall_iso[1]) v = SG::grid(-v + abb_source(a, k, 1, x0 + 1, y, z)); \
                g1[q] = v;                                                              \
            }                                                                           \
        }                                                                               \
    }
    LBPC_Q7(LBPC_AGG)
#undef LBPC_AGG
    const double2 ep = *reinterpret_cast<const double2*>(hp + n0);
    const double e0 = excess_plus<Mode<P>::G>(ep.x, g0), e1 = excess_plus<Mode<P>::G>(ep.y, g1);
    pair_collide<P, FLOW>(a, f0, f1, g0, g1, e0, e1);
    // fresh copies of the indices and bases for the scatter (see opaque())
    int m0 = n0, mdn = dn0, mup = up1, tsy = sy, tsz = sz;
    TF<P>* Fw = F;
    TG<P>* Gw = G;
    opaque(m0); opaque(mdn); opaque(mup); opaque(tsy); opaque(tsz); opaque(Fw); opaque(Gw);
    // ---- scatter ----
    if constexpr (FLOW) {
#define LBPC_ASF(q, ex, ey, ez, op)                                                      \
        {                                                                               \
            const C sh = fshift(k, q);                                                  \
            if constexpr (!ODD) {                                                       \
                *reinterpret_cast<VF*>(Fw + (size_t)op * N + m0) = PRF::enc(f0[q], f1[q], sh); \
            } else {                                                                    \
                const int o2 = (ey) * tsy + (ez) * tsz;                                   \
                TFt* dq = Fw + (size_t)q * N;                                            \
                if constexpr ((ex) == 0) {                                              \
                    *reinterpret_cast<VF*>(dq + m0 + o2) = PRF::enc(f0[q], f1[q], sh);  \
                } else if constexpr ((ex) == 1) {                                       \
                    dq[(m0 + 1) + o2] = SF::enc(f0[q], sh);                             \
                    dq[whi ? ((op) - (q)) * N32 + (m0 + 1) : mup + o2] = SF::enc(f1[q], sh); \
                } else {                                                                \
                    dq[wlo ? ((op) - (q)) * N32 + m0 : mdn + o2] = SF::enc(f0[q], sh);  \
                    dq[m0 + o2] = SF::enc(f1[q], sh);                                   \
                }                                                                       \
            }                                                                           \
        }
        LBPC_Q19(LBPC_ASF)
#undef LBPC_ASF
    }
#define LBPC_ASG(q, ex, ey, ez, op)                                                      \
    {                                                                                   \
        if constexpr (!ODD) {                                                           \
            const VG v = PRG::enc_g(g0[q], g1[q], k.gshift);                            \
            *reinterpret_cast<VG*>(Gw + (size_t)(op - 1) * N + m0) = v;                   \
            PRG::dec(v, k.gshift, g0[q], g1[q]);                                        \
        } else {                                                                        \
            const int o2 = (ey) * tsy + (ez) * tsz;                                       \
            TGt* dq = Gw + (size_t)(q - 1) * N;                                          \
            if constexpr ((ex) == 0) {                                                  \
                const VG v = PRG::enc_g(g0[q], g1[q], k.gshift);                        \
                *reinterpret_cast<VG*>(dq + m0 + o2) = v;                               \
                PRG::dec(v, k.gshift, g0[q], g1[q]);                                    \
            } else if constexpr ((ex) == 1) {                                           \
                const TGt v0 = SG::enc_g(g0[q], k.gshift), v1 = SG::enc_g(g1[q], k.gshift); \
                dq[(m0 + 1) + o2] = v0;                                                 \
                TGt vb = v1;                                                            \
                if (whi && a.wall_iso[1])                                               \
                    vb = SG::enc_g(-SG::dec(v1, k.gshift) + abb_source(a, k, 1, x0 + 1, y, z), k.gshift); \
                dq[whi ? ((op) - (q)) * N32 + (m0 + 1) : mup + o2] = vb;                \
                g0[q] = SG::dec(v0, k.gshift);                                          \
                g1[q] = SG::dec(v1, k.gshift);                                          \
            } else {                                                                    \
                const TGt v0 = SG::enc_g(g0[q], k.gshift), v1 = SG::enc_g(g1[q], k.gshift); \
                TGt vb = v0;                                                            \
                if (wlo && a.wall_iso[0])                                               \
                    vb = SG::enc_g(-SG::dec(v0, k.gshift) + abb_source(a, k, 0, x0, y, z), k.gshift); \
                dq[wlo ? ((op) - (q)) * N32 + m0 : mdn + o2] = vb;                      \
                dq[m0 + o2] = v1;                                                       \
                g0[q] = SG::dec(v0, k.gshift);                                          \
                g1[q] = SG::dec(v1, k.gshift);                                          \
            }                                                                           \
        }                                                                               \
    }
    LBPC_Q7(LBPC_ASG)
#undef LBPC_ASG
    *reinterpret_cast<double2*>(hp + n0) =
        make_double2(excess_minus<Mode<P>::G>(e0, g0), excess_minus<Mode<P>::G>(e1, g1));
}

// Macroscopic state of node n and its contributions to the diagnostics sums
// (acc: sum f_l, sum h, sum rho, -x wall flux, -x wall gradient, non-finite count).
template <int P, int LAYOUT, bool FLOW>
LBPC_HD void macro_node(const Args& a, int n, const TF<P>* fs,
                        const TG<P>* gs, const double* hp, const MacroOut& out,
                        double* acc) {
    using C = CT<P>;
    const Coef<C>& k = coef<C>(a);
    const int x = n % a.nx, y = (n / a.nx) % a.ny, z = n / (a.nx * a.ny);
    const Nb b = make_nb(a, x, y, z);
    C f[19], g[7];
    if constexpr (FLOW) gather_f<Mode<P>::F, LAYOUT, true>(a, b, n, fs, f);
    gather_g<Mode<P>::G, LAYOUT, true>(a, b, n, x, y, z, gs, g);
    const double e = excess_plus<Mode<P>::G>(hp[n], g);
    const double h = a.hs + e;
    double Td, fld;  // reported: the FP64 inversion
    invert_excess(a, e, Td, fld);
    C rho = C(0), ux = C(0), uy = C(0), uz = C(0);
    if constexpr (FLOW) {  // the velocity as the step computes it
        C T, fl, jx, jy, jz, Fx, Fy, Fz;
        invert_excess(a, e, T, fl);
        flow_macro(f, k, T, fl, rho, jx, jy, jz, ux, uy, uz, Fx, Fy, Fz);
    }
    if (out.T) out.T[n] = Td;
    if (out.fl) out.fl[n] = fld;
    if (out.h) out.h[n] = h;
    if (out.rho) out.rho[n] = (double)rho;
    if (out.ux) out.ux[n] = (double)ux;
    if (out.uy) out.uy[n] = (double)uy;
    if (out.uz) out.uz[n] = (double)uz;
    if (acc) {
        acc[0] += fld;
        acc[1] += h;
        acc[2] += (double)rho;
        if (x == 0) {
            const double Tw = a.Tw[0][y + a.ny * z];
            if (a.wall_iso[0]) acc[3] += 2.0 * ((double)g[1] + (double)k.gshift) - (double)k.wT_cref * Tw;
            acc[4] += (Tw - Td) * 2.0;
        }
        const C gsum = ((g[1] + g[2]) + (g[3] + g[4])) + (g[5] + g[6]);
        if (!isfinite(h) || !isfinite((double)rho) || !isfinite((double)gsum)) acc[5] += 1.0;
    }
    if (out.lines && y == a.ny / 2) {
        if (z == a.nz / 4) out.lines[x] = fld;
        if (z == a.nz / 2) out.lines[a.nx + x] = fld;
        if (z == (3 * a.nz) / 4) out.lines[2 * a.nx + x] = fld;
    }
}

// Value of pre-collision population q of node m in the state to load: Q when given,
// else the rest equilibrium of f (rho = 1, u = 0) and g^eq(h0, T(h0), 0) of Eq. 7.
template <class C>
LBPC_HD double state_f(const double* Qf, size_t N, int q, int m) {
    return Qf ? Qf[(size_t)q * N + m] : (q == 0 ? 1.0 / 3.0 : (q < 7 ? 1.0 / 18.0 : 1.0 / 36.0));
}
template <class C>
LBPC_HD double state_g(const Args& a, const Coef<C>& k, const double* Qg, const double* h0,
                       int q, int m) {
    if (Qg) return Qg[(size_t)q * a.N + m];
    C T, fl;
    invert_excess(a, h0[m] - a.hs, T, fl);
    return (double)(k.wa_cref * T);
}

// Write the slots of node (x, y, z) so that a gather in LAYOUT returns the state Q.
// For the pull layout a slot holds the value its downwind neighbour pulls; slots whose
// downwind neighbour lies behind a wall feed the node's own bounce-back.
template <int P, int LAYOUT, bool FLOW>
LBPC_HD void init_node(const Args& a, int x, int y, int z, const double* Qf, const double* Qg,
                       const double* h0, TF<P>* fd, TG<P>* gd) {
    using C = CT<P>;
    const Coef<C>& k = coef<C>(a);
    const int n = x + a.nx * (y + a.ny * z);
    const Nb b = make_nb(a, x, y, z);
    const size_t N = (size_t)a.N;
    if constexpr (FLOW) {
#define LBPC_IF(q, ex, ey, ez, op)                                                       \
        {                                                                               \
            double v;                                                                   \
            if constexpr (LAYOUT == LAYOUT_AA_NATURAL) v = state_f<C>(Qf, N, q, n);     \
            else {                                                                      \
                const bool w = b.template wall<-(ex), -(ey), -(ez)>();                         \
                v = w ? state_f<C>(Qf, N, op, n)                                        \
                      : state_f<C>(Qf, N, q, n + b.template off<-(ex), -(ey), -(ez)>());       \
            }                                                                           \
            fd[(size_t)q * N + n] = Store<Mode<P>::F>::enc((C)(v - (double)fshift(k, q)), C(0)); \
        }
        LBPC_Q19(LBPC_IF)
#undef LBPC_IF
    }
#define LBPC_IG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        double v;                                                                       \
        if constexpr (LAYOUT == LAYOUT_AA_NATURAL) v = state_g(a, k, Qg, h0, q, n);     \
        else {                                                                          \
            const bool w = b.template wall<-(ex), -(ey), -(ez)>();                             \
            if (w) {                                                                    \
                v = state_g(a, k, Qg, h0, op, n);                                       \
                if (a.wall_iso[op - 1])                                                 \
                    v = (double)k.wT_cref * a.Tw[op - 1][face_index(a, op - 1, x, y, z)] - v; \
            } else {                                                                    \
                v = state_g(a, k, Qg, h0, q, n + b.template off<-(ex), -(ey), -(ez)>());       \
            }                                                                           \
        }                                                                               \
        gd[(size_t)(q - 1) * N + n] = Store<Mode<P>::G>::enc_g((C)(v - (double)k.gshift), C(0)); \
    }
    LBPC_Q7(LBPC_IG)
#undef LBPC_IG
}

// e' = h - h_s - sum_a g_a(gathered), so that the stored state reproduces h.
template <int P, int LAYOUT>
LBPC_HD void init_hprime_node(const Args& a, int x, int y, int z, const double* Qg,
                              const double* h0, const TG<P>* gs, double* hp) {
    using C = CT<P>;
    const int n = x + a.nx * (y + a.ny * z);
    const Nb b = make_nb(a, x, y, z);
    double h;
    if (Qg) {
        h = 0.0;
        for (int q = 0; q < 7; q++) h += Qg[(size_t)q * a.N + n];
    } else {
        h = h0[n];
    }
    C g[7];
    gather_g<Mode<P>::G, LAYOUT, true>(a, b, n, x, y, z, gs, g);
    hp[n] = excess_minus<Mode<P>::G>(h - a.hs, g);
}

// Pre-collision populations of node (x, y, z) in FP64 (g_0 = h' = h_s + e').
template <int P, int LAYOUT, bool FLOW>
LBPC_HD void dist_node(const Args& a, int x, int y, int z, const TF<P>* fs,
                       const TG<P>* gs, const double* hp, double* Qf, double* Qg) {
    using C = CT<P>;
    const int n = x + a.nx * (y + a.ny * z);
    const Nb b = make_nb(a, x, y, z);
    const size_t N = (size_t)a.N;
    const Coef<C>& k = coef<C>(a);
    C g[7];
    gather_g<Mode<P>::G, LAYOUT, true>(a, b, n, x, y, z, gs, g);
    const double gs_ = (double)k.gshift;
    Qg[n] = a.hs + hp[n] - 6.0 * gs_;
    for (int q = 1; q < 7; q++) Qg[(size_t)q * N + n] = (double)g[q] + gs_;
    if constexpr (FLOW) {
        if (Qf) {
            C f[19];
            gather_f<Mode<P>::F, LAYOUT, true>(a, b, n, fs, f);
            for (int q = 0; q < 19; q++) Qf[(size_t)q * N + n] = (double)f[q] + (double)fshift(k, q);
        }
    }
}

// ---------------------------------------------------------------------------------
// Adjoint (reverse mode) of one time step.  J = sum f_l(h_N); lambda is the adjoint of
// the pre-collision populations, stored in the natural layout (f: 19 planes, g: 7 planes
// including g_0).  The collision adjoint is evaluated from the macroscopic tape of the
// pre-collision state (d = h - h_s rounded to the compute precision, exactly the value the
// forward inversion used; rho, j), which fixes every nonlinear factor.
// ---------------------------------------------------------------------------------

// Contribution of the adjoint la of an anti-bounce-back population to dJ/dT_w of its wall
// node: omega_T Cp_ref la.  FP64 for FP64 storage; otherwise the FP32 product converted
// exactly by integer operations (the sum over steps stays FP64 without FP64-pipe products
// in the sweep, where the wall lanes' code is predicated in every warp).
LBPC_HD double wall_grad(const Coef<double>& k, double la) { return k.wT_cref * la; }
LBPC_HD double wall_grad(const Coef<float>& k, float la) { return f2d_exact(k.wT_cref * la); }

// Derivatives of the Eq. 2 inversion on the branch the forward took.
template <class C>
LBPC_HD void invert_excess_d(const Coef<C>& k, C d, C& T, C& fl, C& dTde, C& dfde, C& dTdL,
                             C& dfdL) {
    if (d <= C(0)) {
        fl = C(0); T = k.Tm + d * k.Cps_inv;
        dTde = k.Cps_inv; dfde = C(0); dTdL = C(0); dfdL = C(0);
    } else if (d >= k.L) {
        fl = C(1); T = k.Tm + (d - k.L) * k.Cpl_inv;
        dTde = k.Cpl_inv; dfde = C(0); dTdL = -k.Cpl_inv; dfdL = C(0);
    } else {
        fl = d * k.L_inv; T = k.Tm;
        dTde = C(0); dfde = k.L_inv; dTdL = C(0); dfdL = -fl * k.L_inv;
    }
}

// The symmetric D3Q7 relaxation on the six moving populations: out = (I - N^-1 R N) t,
// with t_0 = -sum t_a implied (the same operator acts on deviations in the forward).
template <class C>
LBPC_HD void enth_relax_op(const Coef<C>& k, const C* t, C* out) {
    const C m1 = t[1] - t[2], m2 = t[3] - t[4], m3 = t[5] - t[6];
    const C p12 = t[1] + t[2], p34 = t[3] + t[4], p56 = t[5] + t[6];
    const C S = p12 + p34 + p56;
    const C m5 = C(2) * p12 - (p34 + p56);
    const C m6 = p34 - p56;
    const C A = k.sig4 * S * C(1.0 / 6.0);
    const C B = k.sig5 * m5;
    const C D = k.sig6 * m6 * C(0.25);
    const C hc = C(0.5) * k.sig_chi;
    const C c12 = A + B * C(1.0 / 6.0);
    const C c36 = A - B * C(1.0 / 12.0);
    out[1] = t[1] - (hc * m1 + c12);
    out[2] = t[2] - (-hc * m1 + c12);
    out[3] = t[3] - (hc * m2 + c36 + D);
    out[4] = t[4] - (-hc * m2 + c36 + D);
    out[5] = t[5] - (hc * m3 + c36 - D);
    out[6] = t[6] - (-hc * m3 + c36 - D);
}

// lf[19], lg[7]: in = adjoint of the post-collision populations, out = adjoint of the
// pre-collision populations.  Returns the node's contribution to dJ/dL.
template <class C, bool FLOW>
LBPC_HD C collide_adjoint(const Coef<C>& k, C d, C rho, C jx, C jy, C jz, C* lf, C* lg) {
    C T, fl, dTde, dfde, dTdL, dfdL;
    invert_excess_d(k, d, T, fl, dTde, dfde, dTdL, dfdL);
    C ux = C(0), uy = C(0), uz = C(0), usx = C(0), usy = C(0), usz = C(0), damp = C(0);
    C Fx = C(0), Fy = C(0), Fz = C(0), phi = fl, dphi = C(1);
    if constexpr (FLOW) {
        const C Fb = k.gbeta * (T - k.Tref);
        phi = solid_phi(k, fl, &dphi);
        usx = jx; usy = jy; usz = jz + C(0.5) * Fb;
        damp = C(-2) * (C(1) - phi);
        Fx = damp * usx; Fy = damp * usy; Fz = Fb + damp * usz;
        ux = phi * usx; uy = phi * usy; uz = phi * usz;
    }
    // enthalpy: g*_a = geq_a + K (g - geq)_a (a >= 1), g*_0 = h - sum_a g*_a
    const C lg0 = lg[0];
    C t[7], Kt[7];
    for (int q = 1; q < 7; q++) t[q] = lg[q] - lg0;
    enth_relax_op(k, t, Kt);
    C lgeq[7];
    for (int q = 1; q < 7; q++) lgeq[q] = t[q] - Kt[q];
    const C Cp = fl * k.Cpl + (C(1) - fl) * k.Cps;
    const C lcT = lgeq[1] + lgeq[2] + lgeq[3] + lgeq[4] + lgeq[5] + lgeq[6];
    const C dx = lgeq[1] - lgeq[2], dy = lgeq[3] - lgeq[4], dz = lgeq[5] - lgeq[6];
    const C lvT = ux * dx + uy * dy + uz * dz;
    C lT = k.wa_cref * lcT + C(0.5) * Cp * lvT;
    C lfl = (k.Cpl - k.Cps) * C(0.5) * T * lvT;
    C le = lg0;
    if constexpr (FLOW) {
        const C vT = C(0.5) * Cp * T;
        C lux = vT * dx, luy = vT * dy, luz = vT * dz;
        // mu = diag(1/|row|^2) M lambda*_f (grouped sums as in the forward transform)
        const C* L = lf;
        const C a1 = L[1] + L[2], b1 = L[1] - L[2];
        const C a3 = L[3] + L[4], b3 = L[3] - L[4];
        const C a5 = L[5] + L[6], b5 = L[5] - L[6];
        const C sxy = (L[7] + L[8]) + (L[9] + L[10]);
        const C xy_x = (L[7] - L[8]) + (L[9] - L[10]);
        const C xy_y = (L[7] + L[8]) - (L[9] + L[10]);
        const C xy_p = (L[7] - L[8]) - (L[9] - L[10]);
        const C sxz = (L[11] + L[12]) + (L[13] + L[14]);
        const C xz_x = (L[11] - L[12]) + (L[13] - L[14]);
        const C xz_z = (L[11] + L[12]) - (L[13] + L[14]);
        const C xz_p = (L[11] - L[12]) - (L[13] - L[14]);
        const C syz = (L[15] + L[16]) + (L[17] + L[18]);
        const C yz_y = (L[15] - L[16]) + (L[17] - L[18]);
        const C yz_z = (L[15] + L[16]) - (L[17] + L[18]);
        const C yz_p = (L[15] - L[16]) - (L[17] - L[18]);
        const C sax = a1 + a3 + a5, sdg = sxy + sxz + syz;
        // raw moments R_k = (M lambda*_f)_k; mu_k = R_k / |row k|^2 enters only through the
        // host constants j_s_k = s_k / |row k|^2 and j_h_k = (1 - s_k/2) / |row k|^2
        const C R0 = L[0] + sax + sdg;
        const C R1 = C(-30) * L[0] - C(11) * sax + C(8) * sdg;
        const C R2 = C(12) * L[0] - C(4) * sax + sdg;
        const C tx = xy_x + xz_x, ty = xy_y + yz_y, tz = xz_z + yz_z;
        const C mu3 = (b1 + tx) * C(0.1), mu5 = (b3 + ty) * C(0.1), mu7 = (b5 + tz) * C(0.1);
        const C R4 = tx - C(4) * b1, R6 = ty - C(4) * b3, R8 = tz - C(4) * b5;
        const C a35 = a3 + a5, h9 = (sxy + sxz) - C(2) * syz;
        const C R9 = C(2) * a1 - a35 + h9;
        const C R10 = C(2) * a35 - C(4) * a1 + h9;
        const C k11 = sxy - sxz, a53 = a5 - a3;
        const C R11 = k11 - a53, R12 = C(2) * a53 + k11;
        const C R16 = xy_x - xz_x, R17 = yz_y - xy_y, R18 = xz_z - yz_z;
        // adjoints of m^eq (rate s_k) and of FF (weight 1 - s_k/2)
        const C q1 = k.j_s_e * R1, q2 = k.j_s_eps * R2;
        const C q4 = k.j_s_q * R4, q6 = k.j_s_q * R6, q8 = k.j_s_q * R8;
        const C q9 = k.j_s_nu9 * R9, q10 = k.j_s_pi10 * R10;
        const C q11 = k.j_s_nu11 * R11, q12 = k.j_s_pi12 * R12;
        const C w9 = q9 - C(0.5) * q10, w11 = q11 - C(0.5) * q12;
        const C q13 = k.j_s_nu13 * xy_p, q14 = k.j_s_nu13 * yz_p, q15 = k.j_s_nu13 * xz_p;
        const C r1 = k.j_h_e * R1, r2 = k.j_h_eps * R2;
        const C r4 = k.j_h_q * R4, r6 = k.j_h_q * R6, r8 = k.j_h_q * R8;
        const C v9 = k.j_h_nu9 * R9 - C(0.5) * k.j_h_pi10 * R10;
        const C v11 = k.j_h_nu11 * R11 - C(0.5) * k.j_h_pi12 * R12;
        const C r13 = k.j_h_nu13 * xy_p, r14 = k.j_h_nu13 * yz_p, r15 = k.j_h_nu13 * xz_p;
        const C u2 = ux * ux + uy * uy + uz * uz;
        const C c23 = C(2) / C(3);
        const C lrho = q1 * (C(-11) + C(19) * u2) + q2 * (C(3) - C(5.5) * u2) -
                       c23 * (q4 * ux + q6 * uy + q8 * uz) +
                       w9 * (C(3) * ux * ux - u2) + w11 * (uy * uy - uz * uz) +
                       q13 * ux * uy + q14 * uy * uz + q15 * ux * uz;
        const C cu = C(38) * q1 - C(11) * q2;
        lux += rho * (cu * ux - c23 * q4 + C(4) * w9 * ux + q13 * uy + q15 * uz);
        luy += rho * (cu * uy - c23 * q6 - C(2) * w9 * uy + C(2) * w11 * uy + q13 * ux + q14 * uz);
        luz += rho * (cu * uz - c23 * q8 - C(2) * w9 * uz - C(2) * w11 * uz + q14 * uy + q15 * ux);
        const C cf = C(38) * r1 - C(11) * r2;
        lux += cf * Fx + C(4) * v9 * Fx + r13 * Fy + r15 * Fz;
        luy += cf * Fy - C(2) * v9 * Fy + C(2) * v11 * Fy + r13 * Fx + r14 * Fz;
        luz += cf * Fz - C(2) * v9 * Fz - C(2) * v11 * Fz + r14 * Fy + r15 * Fx;
        const C lFx = cf * ux - c23 * r4 + C(4) * v9 * ux + r13 * uy + r15 * uz + mu3;
        const C lFy = cf * uy - c23 * r6 - C(2) * v9 * uy + C(2) * v11 * uy + r13 * ux + r14 * uz + mu5;
        const C lFz = cf * uz - c23 * r8 - C(2) * v9 * uz - C(2) * v11 * uz + r14 * uy + r15 * ux + mu7;
        // u = phi us, F = F_b z + damp us, us = j + F_b/2 z, F_b = g beta (T - T_ref)
        const C lusx = phi * lux + damp * lFx;
        const C lusy = phi * luy + damp * lFy;
        const C lusz = phi * luz + damp * lFz;
        lfl += dphi * (lux * usx + luy * usy + luz * usz +
                       C(2) * (lFx * usx + lFy * usy + lFz * usz));
        const C lFb = lFz + C(0.5) * lusz;
        lT += k.gbeta * lFb;
        // lambda_f = lambda*_f + M^T lambda_m, lambda_m = (lrho, -s mu, lj, ...), written as
        // M^T (diag(1/|row|^2) R + lambda_m) (M^T diag(1/|row|^2) M = I): lambda*_f is
        // rebuilt from its moments instead of held to the end, and the row-k coefficient
        // (1 - s_k) / |row k|^2 comes from the host; the sums are shared within axis pairs
        // and diagonal quadruples as in the forward
        const C d0 = lrho + R0 * C(1.0 / 19.0), d3 = lusx + mu3, d5 = lusy + mu5, d7 = lusz + mu7;
        const C d1 = k.j_k_e * R1, d2 = k.j_k_eps * R2, d4 = k.j_k_q * R4, d6 = k.j_k_q * R6,
                d8 = k.j_k_q * R8;
        const C d9 = k.j_k_nu9 * R9, d10 = k.j_k_pi10 * R10, d11 = k.j_k_nu11 * R11,
                d12 = k.j_k_pi12 * R12;
        const C d13 = k.j_k_nu13 * xy_p, d14 = k.j_k_nu13 * yz_p, d15 = k.j_k_nu13 * xz_p;
        const C d16 = k.j_k_t * R16, d17 = k.j_k_t * R17, d18 = k.j_k_t * R18;
        lf[0] = d0 - C(30) * d1 + C(12) * d2;
        const C eax = d0 - C(11) * d1 - C(4) * d2;
        const C ox = d3 - C(4) * d4, oy = d5 - C(4) * d6, oz = d7 - C(4) * d8;
        const C ex1 = eax + C(2) * d9 - C(4) * d10;
        const C cyz = eax - d9 + C(2) * d10, w1112 = d11 - C(2) * d12;
        const C ey1 = cyz + w1112, ez1 = cyz - w1112;
        lf[1] = ex1 + ox;
        lf[2] = ex1 - ox;
        lf[3] = ey1 + oy;
        lf[4] = ey1 - oy;
        lf[5] = ez1 + oz;
        lf[6] = ez1 - oz;
        const C edg = d0 + C(8) * d1 + d2;
        const C X = d3 + d4, Y = d5 + d6, Z = d7 + d8;
        const C a910 = edg + d9 + d10, b1112 = d11 + d12;
        const C exy = a910 + b1112, exz = a910 - b1112;
        const C eyz = edg - C(2) * d9 - C(2) * d10;
        {
            const C u = X + d16, v = Y - d17, Pp = exy + d13, Qq = exy - d13;
            const C s = u + v, w = v - u;
            lf[7] = Pp + s;
            lf[8] = Qq + w;
            lf[9] = Qq - w;
            lf[10] = Pp - s;
        }
        {
            const C u = X - d16, v = Z + d18, Pp = exz + d15, Qq = exz - d15;
            const C s = u + v, w = v - u;
            lf[11] = Pp + s;
            lf[12] = Qq + w;
            lf[13] = Qq - w;
            lf[14] = Pp - s;
        }
        {
            const C u = Y + d17, v = Z - d18, Pp = eyz + d14, Qq = eyz - d14;
            const C s = u + v, w = v - u;
            lf[15] = Pp + s;
            lf[16] = Qq + w;
            lf[17] = Qq - w;
            lf[18] = Pp - s;
        }
    }
    le += lT * dTde + lfl * dfde;
    lg[0] = le;
    for (int q = 1; q < 7; q++) lg[q] = Kt[q] + le;
    return lT * dTdL + lfl * dfdL;
}

// Adjoint seed at the final state: lambda_g = d f_l / dh on every g population,
// lambda_f = 0; returns d f_l / dL and writes f_l (for J).
template <int P, bool FLOW>
LBPC_HD CT<P> adj_seed_node(const Args& a, int x, int y, int z,
                                           const TG<P>* gs, const double* hp,
                                           CT<P>* lam, double& fl_out) {
    using C = CT<P>;
    const Coef<C>& k = coef<C>(a);
    const int n = x + a.nx * (y + a.ny * z);
    const Nb b = make_nb(a, x, y, z);
    C g[7];
    gather_g<Mode<P>::G, LAYOUT_PULL, true>(a, b, n, x, y, z, gs, g);
    const double e = excess_plus<Mode<P>::G>(hp[n], g);
    C T, fl, dTde, dfde, dTdL, dfdL;
    invert_excess_d(k, tape_excess(a, e, C(0)), T, fl, dTde, dfde, dTdL, dfdL);
    const size_t N = (size_t)a.N;
    const int nf = FLOW ? 19 : 0;
    for (int q = 0; q < nf; q++) lam[(size_t)q * N + n] = C(0);
    for (int q = 0; q < 7; q++) lam[(size_t)(nf + q) * N + n] = dfde;
    fl_out = (double)fl;
    return dfdL;
}

// One reverse step of node y: transposed stream (gather of lambda_{n+1} from the
// downwind neighbours, with the transposed wall rules) then transposed collision with
// the tape of step n.  Accumulates dJ/dT_w of face `wface` and returns the dJ/dL part.
template <int P, bool FLOW, class NB>
LBPC_HD CT<P> adj_reverse_node(const Args& a, const NB& b, int x, int y, int z,
                                              const CT<P>* lin,
                                              CT<P>* lout, const CT<P>* tape_e,
                                              const CT<P>* tape_m, int wface,
                                              double* gtw) {
    using C = CT<P>;
    const Coef<C>& k = coef<C>(a);
    const int n = x + a.nx * (y + a.ny * z);
    const size_t N = (size_t)a.N;
    constexpr int nf = FLOW ? 19 : 0;
    C lf[19], lg[7];
    if constexpr (FLOW) {
#define LBPC_AF(q, ex, ey, ez, op)                                                       \
        {                                                                               \
            const bool w = b.template wall<-(ex), -(ey), -(ez)>();                      \
            lf[q] = w ? lin[(size_t)op * N + n]                                         \
                      : lin[(size_t)q * N + n + b.template off<-(ex), -(ey), -(ez)>()];  \
        }
        LBPC_Q19(LBPC_AF)
#undef LBPC_AF
    }
    lg[0] = lin[(size_t)nf * N + n];
#define LBPC_AG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        const bool w = b.template wall<-(ex), -(ey), -(ez)>();                          \
        if (w) {                                                                        \
            const C la = lin[(size_t)(nf + op) * N + n];                                \
            if (a.wall_iso[op - 1]) {                                                   \
                lg[q] = -la;                                                            \
                if (op - 1 == wface)                                                    \
                    gtw[face_index(a, op - 1, x, y, z)] += wall_grad(k, la);            \
            } else {                                                                    \
                lg[q] = la;                                                             \
            }                                                                           \
        } else {                                                                        \
            lg[q] = lin[(size_t)(nf + q) * N + n + b.template off<-(ex), -(ey), -(ez)>()]; \
        }                                                                               \
    }
    LBPC_Q7(LBPC_AG)
#undef LBPC_AG
    C rho = C(0), jx = C(0), jy = C(0), jz = C(0);
    if constexpr (FLOW) {
        rho = tape_m[n];
        jx = tape_m[N + n];
        jy = tape_m[2 * N + n];
        jz = tape_m[3 * N + n];
    }
    const C dL = collide_adjoint<C, FLOW>(k, tape_e[n], rho, jx, jy, jz, lf, lg);
    for (int q = 0; q < nf; q++) lout[(size_t)q * N + n] = lf[q];
    for (int q = 0; q < 7; q++) lout[(size_t)(nf + q) * N + n] = lg[q];
    return dL;
}

// Reverse step of two nodes (x0, x0 + 1) of a row away from every y and z face (even nx):
// lambda_q of node x is lambda_{n+1} in plane q at x + e_q, or the reflected plane at x
// when x + e_q lies behind an x wall; every other access is an aligned pair.
template <int P, bool FLOW>
LBPC_HD CT<P> adj_reverse_pair(const Args& a, int x0, int y, int z, const CT<P>* lin,
                               CT<P>* lout, const CT<P>* tape_e, const CT<P>* tape_m,
                               int wface, double* gtw) {
    using C = CT<P>;
    using VC = typename Vec2<C>::type;
    const Coef<C>& k = coef<C>(a);
    const size_t N = (size_t)a.N;
    const int N32 = a.N;  // 3 N < 2^31 (kPairMaxN)
    constexpr int nf = FLOW ? 19 : 0;
    const int sy = a.nx, sz = a.nx * a.ny;
    const int n0 = x0 + a.nx * (y + a.ny * z), n1 = n0 + 1;
    const bool xlo = x0 == 0, xhi = x0 + 1 == a.nx - 1;
    const bool wlo = xlo && a.wall[0], whi = xhi && a.wall[1];
    const int dn0 = xlo ? n0 + a.nx - 1 : n0 - 1;    // x0 - 1 (wrapped)
    const int up1 = xhi ? n1 - (a.nx - 1) : n1 + 1;  // x1 + 1 (wrapped)
    C lf0[19], lf1[19], lg0[7], lg1[7];
    if constexpr (FLOW) {
#define LBPC_RF(q, ex, ey, ez, op)                                                       \
        {                                                                               \
            const int o = (ey) * sy + (ez) * sz;                                        \
            const C* pl = lin + (size_t)q * N;                                          \
            if constexpr ((ex) == 0) {                                                  \
                const VC v = ld_any<true>(reinterpret_cast<const VC*>(pl + n0 + o));    \
                lf0[q] = v.x; lf1[q] = v.y;                                             \
            } else if constexpr ((ex) == 1) {                                           \
                lf0[q] = ld_any<true>(pl + n1 + o);                                     \
                lf1[q] = ld_any<true>(pl + (whi ? ((op) - (q)) * N32 + n1 : up1 + o)); \
            } else {                                                                    \
                lf0[q] = ld_any<true>(pl + (wlo ? ((op) - (q)) * N32 + n0 : dn0 + o)); \
                lf1[q] = ld_any<true>(pl + n0 + o);                                     \
            }                                                                           \
        }
        LBPC_Q19(LBPC_RF)
#undef LBPC_RF
    }
    {
        const VC v = ld_any<true>(reinterpret_cast<const VC*>(lin + (size_t)nf * N + n0));
        lg0[0] = v.x; lg1[0] = v.y;
    }
#define LBPC_RG(q, ex, ey, ez, op)                                                       \
    {                                                                                   \
        const int o = (ey) * sy + (ez) * sz;                                            \
        const C* pl = lin + (size_t)(nf + q) * N;                                       \
        if constexpr ((ex) == 0) {                                                      \
            const VC v = ld_any<true>(reinterpret_cast<const VC*>(pl + n0 + o));        \
            lg0[q] = v.x; lg1[q] = v.y;                                                 \
        } else if constexpr ((ex) == 1) {                                               \
            lg0[q] = ld_any<true>(pl + n1 + o);                                         \
            const C la = ld_any<true>(pl + (whi ? ((op) - (q)) * N32 + n1 : up1 + o));  \
            const bool iso = whi && a.wall_iso[1];                                      \
            lg1[q] = iso ? -la : la;                                                    \
            if (iso && wface == 1) gtw[y + a.ny * z] += wall_grad(k, la);          \
        } else {                                                                        \
            const C la = ld_any<true>(pl + (wlo ? ((op) - (q)) * N32 + n0 : dn0 + o));  \
            const bool iso = wlo && a.wall_iso[0];                                      \
            lg0[q] = iso ? -la : la;                                                    \
            if (iso && wface == 0) gtw[y + a.ny * z] += wall_grad(k, la);          \
            lg1[q] = ld_any<true>(pl + n0 + o);                                         \
        }                                                                               \
    }
    LBPC_Q7(LBPC_RG)
#undef LBPC_RG
    C r0 = C(0), jx0 = C(0), jy0 = C(0), jz0 = C(0), r1 = C(0), jx1 = C(0), jy1 = C(0), jz1 = C(0);
    if constexpr (FLOW) {
        VC v = ld_any<true>(reinterpret_cast<const VC*>(tape_m + n0));
        r0 = v.x; r1 = v.y;
        v = ld_any<true>(reinterpret_cast<const VC*>(tape_m + N + n0));
        jx0 = v.x; jx1 = v.y;
        v = ld_any<true>(reinterpret_cast<const VC*>(tape_m + 2 * N + n0));
        jy0 = v.x; jy1 = v.y;
        v = ld_any<true>(reinterpret_cast<const VC*>(tape_m + 3 * N + n0));
        jz0 = v.x; jz1 = v.y;
    }
    const VC d = ld_any<true>(reinterpret_cast<const VC*>(tape_e + n0));
    const C dL = collide_adjoint<C, FLOW>(k, d.x, r0, jx0, jy0, jz0, lf0, lg0) +
                 collide_adjoint<C, FLOW>(k, d.y, r1, jx1, jy1, jz1, lf1, lg1);
    for (int q = 0; q < nf; q++)
        *reinterpret_cast<VC*>(lout + (size_t)q * N + n0) = VC{lf0[q], lf1[q]};
    for (int q = 0; q < 7; q++)
        *reinterpret_cast<VC*>(lout + (size_t)(nf + q) * N + n0) = VC{lg0[q], lg1[q]};
    return dL;
}

#if defined(__CUDACC__)
// ---------------------------------------------------------------------------------
// Kernels: one thread per node on a (x-block, y-block, z) grid.
// ---------------------------------------------------------------------------------
#define LBPC_NODE_XYZ                                                                    \
    const int x = blockIdx.x * blockDim.x + threadIdx.x;                                \
    const int y = blockIdx.y * blockDim.y + threadIdx.y;                                \
    const int z = blockIdx.z;                                                           \
    if (x >= a.nx || y >= a.ny) return;

// One node per thread; with TAPE (pull) also the adjoint tape.
template <int P, int KIND, int FLOW, bool TAPE>
__global__ void __launch_bounds__(STEP_THREADS)
k_step(const __grid_constant__ Args a, const TF<P>* fs, TF<P>* fd,
       const TG<P>* gs, TG<P>* gd, double* __restrict__ hp, CT<P>* __restrict__ tape_e,
       CT<P>* __restrict__ tape_m) {
    LBPC_NODE_XYZ
    step_node<P, KIND, FLOW, TAPE>(a, x, y, z, fs, fd, gs, gd, hp, tape_e, tape_m);
}


// Pull step, two nodes per thread along x (even nx).  Warps whose rows all lie away
// from the y and z faces take the paired path; others run the per-node path twice.
// With TAPE also the adjoint tape.  Blocks per SM: FP32 five (96 registers), four when
// taping; 16-bit f (collision rebuilt from the moments) six (80 registers), five when taping.
template <int P, int FLOW, bool TAPE>
__global__ void __launch_bounds__(STEP_THREADS, TAPE ? (kRebuild<P> ? 5 : 4) : (kRebuild<P> ? 6 : 5))
k_step_pull_x2(const __grid_constant__ Args a, const TF<P>* fs,
               TF<P>* fd, const TG<P>* gs, TG<P>* gd,
               double* __restrict__ hp, CT<P>* __restrict__ tape_e,
               CT<P>* __restrict__ tape_m) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool valid = x0 < a.nx && y < a.ny;
    const bool inner = !valid || (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1);
    const bool paired = __all_sync(0xffffffffu, inner);
    if (!valid) return;
    if (paired) {
        step_pair_pull<P, FLOW, TAPE>(a, x0, y, z, fs, fd, gs, gd, hp, tape_e, tape_m);
    } else {
        step_node<P, STEP_PULL, FLOW, TAPE>(a, x0, y, z, fs, fd, gs, gd, hp, tape_e, tape_m);
        step_node<P, STEP_PULL, FLOW, TAPE>(a, x0 + 1, y, z, fs, fd, gs, gd, hp, tape_e, tape_m);
    }
}


// AA step, two nodes per thread along x (even nx); same vote as the pull pair kernel.
// Five blocks per SM (96 registers; a few bytes of spills in some variants); the even step
// with 16-bit f six (80 registers; the odd step spills at six).
template <int P, int FLOW, bool ODD>
__global__ void __launch_bounds__(STEP_THREADS, kRebuild<P> && !ODD ? 6 : 5)
k_step_aa_x2(const __grid_constant__ Args a, TF<P>* F, TG<P>* G, double* __restrict__ hp) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool valid = x0 < a.nx && y < a.ny;
    const bool inner = !valid || (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1);
    const bool paired = __all_sync(0xffffffffu, inner);
    if (!valid) return;
    constexpr int KIND = ODD ? STEP_AA_ODD : STEP_AA_EVEN;
    if (paired) {
        step_pair_aa<P, FLOW, ODD>(a, x0, y, z, F, G, hp);
    } else {
        step_node<P, KIND, FLOW>(a, x0, y, z, F, F, G, G, hp);
        step_node<P, KIND, FLOW>(a, x0 + 1, y, z, F, F, G, G, hp);
    }
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Macroscopic fields of the current state and FP64 block partial sums for diagnostics
// (grid-stride over nodes; one partial row per block, summed later in a fixed order).
template <int P, int LAYOUT, bool FLOW>
__global__ void __launch_bounds__(RED_THREADS)
k_macro(const __grid_constant__ Args a, const TF<P>* __restrict__ fs,
        const TG<P>* __restrict__ gs, const double* __restrict__ hp,
        const MacroOut out) {
    double acc[NRED] = {0, 0, 0, 0, 0, 0};
    // 64-bit loop index: n + stride may pass 2^31 - 1 near the node limit
    for (long long n = blockIdx.x * blockDim.x + threadIdx.x; n < a.N;
         n += (long long)gridDim.x * blockDim.x)
        macro_node<P, LAYOUT, FLOW>(a, (int)n, fs, gs, hp, out, out.partial ? acc : nullptr);
    if (!out.partial) return;
    __shared__ double sh[RED_THREADS / 32][NRED];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NRED; i++) {
        const double v = warp_sum(acc[i]);
        if (lane == 0) sh[wid][i] = v;
    }
    __syncthreads();
    if (threadIdx.x < NRED) {
        double s = 0.0;
        for (int w = 0; w < RED_THREADS / 32; w++) s += sh[w][threadIdx.x];
        out.partial[blockIdx.x * NRED + threadIdx.x] = s;
    }
}

template <int P, int LAYOUT, bool FLOW>
__global__ void __launch_bounds__(STEP_THREADS)
k_init(const __grid_constant__ Args a, const double* __restrict__ Qf, const double* __restrict__ Qg,
       const double* __restrict__ h0, TF<P>* fd, TG<P>* gd) {
    LBPC_NODE_XYZ
    init_node<P, LAYOUT, FLOW>(a, x, y, z, Qf, Qg, h0, fd, gd);
}

template <int P, int LAYOUT>
__global__ void __launch_bounds__(STEP_THREADS)
k_init_hprime(const __grid_constant__ Args a, const double* __restrict__ Qg,
              const double* __restrict__ h0, const TG<P>* __restrict__ gs,
              double* __restrict__ hp) {
    LBPC_NODE_XYZ
    init_hprime_node<P, LAYOUT>(a, x, y, z, Qg, h0, gs, hp);
}

template <int P, int LAYOUT, bool FLOW>
__global__ void __launch_bounds__(STEP_THREADS)
k_dist(const __grid_constant__ Args a, const TF<P>* __restrict__ fs,
       const TG<P>* __restrict__ gs, const double* __restrict__ hp,
       double* __restrict__ Qf, double* __restrict__ Qg) {
    LBPC_NODE_XYZ
    dist_node<P, LAYOUT, FLOW>(a, x, y, z, fs, gs, hp, Qf, Qg);
}


// Divergence check between steps: sets *flag when a stored g population (any of the six
// planes, any layout) or the FP64 rest channel is not finite, by tests on the bits (all
// exponent bits set).  A non-finite f reaches g within one step through u.
template <class T> __device__ __forceinline__ bool nonfinite_bits(T v);
template <> __device__ __forceinline__ bool nonfinite_bits<double>(double v) {
    return ((__double_as_longlong(v) >> 52) & 0x7ff) == 0x7ff;
}
template <> __device__ __forceinline__ bool nonfinite_bits<float>(float v) {
    return (__float_as_uint(v) & 0x7f800000u) == 0x7f800000u;
}
template <> __device__ __forceinline__ bool nonfinite_bits<__half>(__half v) {
    return (__half_as_ushort(v) & 0x7c00u) == 0x7c00u;
}
template <> __device__ __forceinline__ bool nonfinite_bits<__nv_bfloat16>(__nv_bfloat16 v) {
    return (__bfloat16_as_ushort(v) & 0x7f80u) == 0x7f80u;
}
template <int P>
__global__ void __launch_bounds__(256)
k_check(const __grid_constant__ Args a, const TG<P>* __restrict__ g,
        const double* __restrict__ hp, int* flag) {
    int bad = 0;
    const size_t N = (size_t)a.N;
    for (long long n = blockIdx.x * blockDim.x + threadIdx.x; n < a.N;
         n += (long long)gridDim.x * blockDim.x) {
        bad |= nonfinite_bits(hp[n]);
#pragma unroll
        for (int q = 0; q < 6; q++) bad |= nonfinite_bits(g[(size_t)q * N + n]);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1;
}

// ---- adjoint kernels ----
// Sum of v over the block (STEP_THREADS threads), valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[STEP_THREADS / 32];
    v = warp_sum(v);
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
    if ((tid & 31) == 0) sh[tid >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (tid == 0)
        for (int w = 0; w < STEP_THREADS / 32; w++) s += sh[w];
    return s;
}

__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// Per-warp slot of the adjoint's dJ/dL partials (ADJ_WARPS_PER_BLOCK per block).
static_assert(STEP_THREADS / 32 == ADJ_WARPS_PER_BLOCK, "one partial slot per warp");
__device__ __forceinline__ int warp_slot() {
    return block_linear() * ADJ_WARPS_PER_BLOCK + ((threadIdx.x + blockDim.x * threadIdx.y) >> 5);
}

template <int P, bool FLOW>
__global__ void __launch_bounds__(STEP_THREADS)
k_adj_seed(const __grid_constant__ Args a, const TG<P>* __restrict__ gs,
           const double* __restrict__ hp, CT<P>* __restrict__ lam,
           double* __restrict__ Lpart, double* __restrict__ Jpart) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    double dL = 0.0, fl = 0.0;
    if (x < a.nx && y < a.ny) dL = (double)adj_seed_node<P, FLOW>(a, x, y, z, gs, hp, lam, fl);
    const double wL = warp_sum(dL);
    if (((threadIdx.x + blockDim.x * threadIdx.y) & 31) == 0) Lpart[warp_slot()] = wL;
    const double sJ = block_sum(fl);
    if (threadIdx.x == 0 && threadIdx.y == 0) Jpart[block_linear()] = sJ;
}

template <int P, bool FLOW>
__global__ void __launch_bounds__(STEP_THREADS)
k_adj_reverse(const __grid_constant__ Args a, const CT<P>* __restrict__ lin,
              CT<P>* __restrict__ lout, const CT<P>* __restrict__ tape_e,
              const CT<P>* __restrict__ tape_m, int wface, double* gtw,
              double* __restrict__ Lpart) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    CT<P> dL = CT<P>(0);
    if (x < a.nx && y < a.ny) {
        if (is_interior(a, x, y, z))
            dL = adj_reverse_node<P, FLOW>(a, NbInterior{a.nx, a.nx * a.ny}, x, y, z, lin, lout,
                                           tape_e, tape_m, wface, gtw);
        else
            dL = adj_reverse_node<P, FLOW>(a, make_nb(a, x, y, z), x, y, z, lin, lout, tape_e,
                                           tape_m, wface, gtw);
    }
    // warp partials only (no block barrier in the reverse sweep), summed within the warp in
    // the compute precision and accumulated over warps and steps in FP64
    const CT<P> w = warp_sum(dL);
    if (((threadIdx.x + blockDim.x * threadIdx.y) & 31) == 0) Lpart[warp_slot()] += (double)w;
}

// Reverse step, two nodes per thread along x (even nx); the pull kernels' vote.  Five
// blocks per SM (96 registers, no spills).
template <int P, bool FLOW>
__global__ void __launch_bounds__(STEP_THREADS, 5)
k_adj_reverse_x2(const __grid_constant__ Args a, const CT<P>* __restrict__ lin,
                 CT<P>* __restrict__ lout, const CT<P>* __restrict__ tape_e,
                 const CT<P>* __restrict__ tape_m, int wface, double* gtw,
                 double* __restrict__ Lpart) {
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    const bool valid = x0 < a.nx && y < a.ny;
    const bool inner = !valid || (y > 0 && y < a.ny - 1 && z > 0 && z < a.nz - 1);
    const bool paired = __all_sync(0xffffffffu, inner);
    CT<P> dL = CT<P>(0);
    if (valid) {
        if (paired) {
            dL = adj_reverse_pair<P, FLOW>(a, x0, y, z, lin, lout, tape_e, tape_m, wface, gtw);
        } else {
            for (int x = x0; x < x0 + 2; x++)
                dL += adj_reverse_node<P, FLOW>(a, make_nb(a, x, y, z), x, y, z, lin, lout, tape_e,
                                                tape_m, wface, gtw);
        }
    }
    // warp partials in the compute precision, accumulated in FP64 (see k_adj_reverse)
    const CT<P> w = warp_sum(dL);
    if (((threadIdx.x + blockDim.x * threadIdx.y) & 31) == 0) Lpart[warp_slot()] += (double)w;
}

// ---------------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------------
inline dim3 node_block(const Args& a) { return node_block_dims(a.nx); }
inline dim3 node_grid(const Args& a, dim3 blk) {
    return dim3((a.nx + blk.x - 1) / blk.x, (a.ny + blk.y - 1) / blk.y, a.nz);
}

template <int P>
struct Impl {
    using T = TF<P>;
    using TGp = TG<P>;

    // TAPE (pull only): also write the adjoint tape of this step to tape_e / tape_m
    template <int KIND, int FLOW, bool TAPE = false>
    static void step_k(const Args& a, const void* fs, void* fd, const void* gs, void* gd,
                       double* hp, cudaStream_t s, void* tape_e = nullptr,
                       void* tape_m = nullptr) {
        using C = CT<P>;
        if constexpr (P != LBPC_FP64) {  // FP64 keeps one node per thread
            if (a.nx % 2 == 0 && a.N <= kPairMaxN) {
                const int pairs = a.nx / 2;
                const dim3 blk = node_block_dims(pairs);
                const dim3 grd((pairs + blk.x - 1) / blk.x, (a.ny + blk.y - 1) / blk.y, a.nz);
                if constexpr (KIND == STEP_PULL)
                    k_step_pull_x2<P, FLOW, TAPE><<<grd, blk, 0, s>>>(a, (const T*)fs, (T*)fd,
                                                                (const TGp*)gs, (TGp*)gd, hp,
                                                                (C*)tape_e, (C*)tape_m);
                else
                    k_step_aa_x2<P, FLOW, KIND == STEP_AA_ODD><<<grd, blk, 0, s>>>(a, (T*)fd,
                                                                               (TGp*)gd, hp);
                return;
            }
        }
        const dim3 blk = node_block(a), grd = node_grid(a, blk);
        k_step<P, KIND, FLOW, TAPE><<<grd, blk, 0, s>>>(a, (const T*)fs, (T*)fd, (const TGp*)gs, (TGp*)gd, hp,
                                                  (C*)tape_e, (C*)tape_m);
    }
    static void step(const Args& a, StepKind kind, const void* fs, void* fd, const void* gs,
                     void* gd, double* hp, cudaStream_t s) {
        if (a.flow) {
            if (coef<CT<P>>(a).darcy) {
                if (kind == STEP_PULL) step_k<STEP_PULL, 2>(a, fs, fd, gs, gd, hp, s);
                else if (kind == STEP_AA_EVEN) step_k<STEP_AA_EVEN, 2>(a, fs, fd, gs, gd, hp, s);
                else step_k<STEP_AA_ODD, 2>(a, fs, fd, gs, gd, hp, s);
            } else {
                if (kind == STEP_PULL) step_k<STEP_PULL, 1>(a, fs, fd, gs, gd, hp, s);
                else if (kind == STEP_AA_EVEN) step_k<STEP_AA_EVEN, 1>(a, fs, fd, gs, gd, hp, s);
                else step_k<STEP_AA_ODD, 1>(a, fs, fd, gs, gd, hp, s);
            }
        } else {
            if (kind == STEP_PULL) step_k<STEP_PULL, 0>(a, fs, fd, gs, gd, hp, s);
            else if (kind == STEP_AA_EVEN) step_k<STEP_AA_EVEN, 0>(a, fs, fd, gs, gd, hp, s);
            else step_k<STEP_AA_ODD, 0>(a, fs, fd, gs, gd, hp, s);
        }
    }

    template <int LAYOUT, bool FLOW>
    static void macro_k(const Args& a, const void* f, const void* g, const double* hp,
                        const MacroOut& o, cudaStream_t s) {
        k_macro<P, LAYOUT, FLOW><<<RED_BLOCKS, RED_THREADS, 0, s>>>(a, (const T*)f, (const TGp*)g, hp, o);
    }
    static void macro(const Args& a, Layout lay, const void* f, const void* g, const double* hp,
                      const MacroOut& o, cudaStream_t s) {
        if (a.flow) {
            if (lay == LAYOUT_PULL) macro_k<LAYOUT_PULL, true>(a, f, g, hp, o, s);
            else if (lay == LAYOUT_AA_NATURAL) macro_k<LAYOUT_AA_NATURAL, true>(a, f, g, hp, o, s);
            else macro_k<LAYOUT_AA_SWAPPED, true>(a, f, g, hp, o, s);
        } else {
            if (lay == LAYOUT_PULL) macro_k<LAYOUT_PULL, false>(a, f, g, hp, o, s);
            else if (lay == LAYOUT_AA_NATURAL) macro_k<LAYOUT_AA_NATURAL, false>(a, f, g, hp, o, s);
            else macro_k<LAYOUT_AA_SWAPPED, false>(a, f, g, hp, o, s);
        }
    }

    static void init(const Args& a, Layout lay, const double* Qf, const double* Qg,
                     const double* h0, void* f, void* g, double* hp, cudaStream_t s) {
        const dim3 blk = node_block(a), grd = node_grid(a, blk);
        if (lay == LAYOUT_PULL) {
            if (a.flow) k_init<P, LAYOUT_PULL, true><<<grd, blk, 0, s>>>(a, Qf, Qg, h0, (T*)f, (TGp*)g);
            else k_init<P, LAYOUT_PULL, false><<<grd, blk, 0, s>>>(a, Qf, Qg, h0, (T*)f, (TGp*)g);
            k_init_hprime<P, LAYOUT_PULL><<<grd, blk, 0, s>>>(a, Qg, h0, (const TGp*)g, hp);
        } else {
            if (a.flow) k_init<P, LAYOUT_AA_NATURAL, true><<<grd, blk, 0, s>>>(a, Qf, Qg, h0, (T*)f, (TGp*)g);
            else k_init<P, LAYOUT_AA_NATURAL, false><<<grd, blk, 0, s>>>(a, Qf, Qg, h0, (T*)f, (TGp*)g);
            k_init_hprime<P, LAYOUT_AA_NATURAL><<<grd, blk, 0, s>>>(a, Qg, h0, (const TGp*)g, hp);
        }
    }

    template <int LAYOUT>
    static void dist_k(const Args& a, const void* f, const void* g, const double* hp,
                       double* Qf, double* Qg, cudaStream_t s) {
        const dim3 blk = node_block(a), grd = node_grid(a, blk);
        if (a.flow) k_dist<P, LAYOUT, true><<<grd, blk, 0, s>>>(a, (const T*)f, (const TGp*)g, hp, Qf, Qg);
        else k_dist<P, LAYOUT, false><<<grd, blk, 0, s>>>(a, (const T*)f, (const TGp*)g, hp, Qf, Qg);
    }
    static void dist(const Args& a, Layout lay, const void* f, const void* g, const double* hp,
                     double* Qf, double* Qg, cudaStream_t s) {
        if (lay == LAYOUT_PULL) dist_k<LAYOUT_PULL>(a, f, g, hp, Qf, Qg, s);
        else if (lay == LAYOUT_AA_NATURAL) dist_k<LAYOUT_AA_NATURAL>(a, f, g, hp, Qf, Qg, s);
        else dist_k<LAYOUT_AA_SWAPPED>(a, f, g, hp, Qf, Qg, s);
    }

    static void step_tape(const Args& a, const void* fs, void* fd, const void* gs, void* gd,
                          double* hp, void* tape_e, void* tape_m, cudaStream_t s) {
        if (a.flow && coef<CT<P>>(a).darcy)
            step_k<STEP_PULL, 2, true>(a, fs, fd, gs, gd, hp, s, tape_e, tape_m);
        else if (a.flow)
            step_k<STEP_PULL, 1, true>(a, fs, fd, gs, gd, hp, s, tape_e, tape_m);
        else
            step_k<STEP_PULL, 0, true>(a, fs, fd, gs, gd, hp, s, tape_e, tape_m);
    }
    static void adj_seed(const Args& a, const void* gs, const double* hp, void* lam,
                         double* Lpart, double* Jpart, cudaStream_t s) {
        const dim3 blk = node_block(a), grd = node_grid(a, blk);
        using C = CT<P>;
        if (a.flow) k_adj_seed<P, true><<<grd, blk, 0, s>>>(a, (const TGp*)gs, hp, (C*)lam, Lpart, Jpart);
        else k_adj_seed<P, false><<<grd, blk, 0, s>>>(a, (const TGp*)gs, hp, (C*)lam, Lpart, Jpart);
    }
    static void adj_reverse(const Args& a, const void* lin, void* lout, const void* tape_e,
                            const void* tape_m, int wface, double* gtw, double* Lpart,
                            cudaStream_t s) {
        using C = CT<P>;
        if constexpr (P != LBPC_FP64) {
            // the paired grid never has more blocks than the per-node one that sized Lpart
            if (a.nx % 2 == 0 && a.N <= kPairMaxN) {
                const int pairs = a.nx / 2;
                const dim3 blk = node_block_dims(pairs);
                const dim3 grd((pairs + blk.x - 1) / blk.x, (a.ny + blk.y - 1) / blk.y, a.nz);
                if (a.flow)
                    k_adj_reverse_x2<P, true><<<grd, blk, 0, s>>>(a, (const C*)lin, (C*)lout,
                                                                 (const C*)tape_e, (const C*)tape_m,
                                                                 wface, gtw, Lpart);
                else
                    k_adj_reverse_x2<P, false><<<grd, blk, 0, s>>>(a, (const C*)lin, (C*)lout,
                                                                  (const C*)tape_e,
                                                                  (const C*)tape_m, wface, gtw,
                                                                  Lpart);
                return;
            }
        }
        const dim3 blk = node_block(a), grd = node_grid(a, blk);
        if (a.flow)
            k_adj_reverse<P, true><<<grd, blk, 0, s>>>(a, (const C*)lin, (C*)lout, (const C*)tape_e,
                                                       (const C*)tape_m, wface, gtw, Lpart);
        else
            k_adj_reverse<P, false><<<grd, blk, 0, s>>>(a, (const C*)lin, (C*)lout, (const C*)tape_e,
                                                        (const C*)tape_m, wface, gtw, Lpart);
    }

    static void check(const Args& a, const void* g, const double* hp, int* flag,
                      cudaStream_t s) {
        k_check<P><<<RED_BLOCKS, 256, 0, s>>>(a, (const TGp*)g, hp, flag);
    }

    static const Launchers& table() {
        static const Launchers L = {&step, &macro, &init, &dist, &step_tape, &adj_seed,
                                    &adj_reverse, &check, sizeof(T), sizeof(TGp),
                                    sizeof(CT<P>)};
        return L;
    }
};
#endif  // __CUDACC__

}  // namespace lbpc
