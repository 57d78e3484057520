// Exact projection of a coordinate to its tile index, floor(RN(v * s))
// (Alg. 1 project(); Sect. 3.2), for the CUDA kernels of this library.
#pragma once

namespace raster {

// Projection parameters derived once on the host from the scale s.
struct ProjParams {
    unsigned long long s_odd;  // odd part of the significand of s
    int s_exp;                 // s = s_odd * 2^s_exp
    int s_bits;                // bit length of s_odd
    int d0;                    // 1075 - s_exp: v*s = P * 2^-(d0 - e) for v of biased exponent e
    int top;                   // 52 + s_bits: P = significand(v) * s_odd has top or top+1 bits
    double scale;              // s itself, for the rare FP64 path
};

// Rare path: the definition itself on the FP64 pipe.
static __device__ __noinline__ bool project_coord_fp64(double v, double scale, int* out) {
    double f = floor(__dmul_rn(v, scale));
    if (!(f >= -2147483647.0 && f <= 2147483646.0)) return false;
    *out = (int)f;
    return true;
}

// floor(RN(v * s)) for one coordinate, exactly.
//
// With P = significand(v) * s_odd (exact) and v*s = P * 2^-D, let F = floor(P * 2^-D)
// and let r be the number of bits of P below its 53 leading ones (the rounding
// position, so ulp = 2^(r-D)).  For a result inside the int32 tile range, ulp < 1,
// F and F+1 are representable, and F+1 has an even significand; hence
//   floor(RN(v*s)) = F + 1  iff  (F + 1) - v*s <= ulp/2    (ties round up to F+1),
//   ceil (RN(v*s)) = F + 1  iff  v*s - F       >  ulp/2    (ties round down to F),
// which is one add of a bias before the shift: (P + bias) >> D.  The first
// gives the tile of a positive coordinate, minus the second that of a negative
// one.  NARROW (s_odd below 2^10, every integer precision 0..4) keeps P below
// 2^63; otherwise the 128-bit product is rounded explicitly.
template <bool WIDE>
__device__ __forceinline__ bool project_coord(double v, const ProjParams& pp, int* out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned int e = (unsigned int)(b >> 52) & 0x7FFu;
    if (e - 1u >= 0x7FEu) {  // zero, subnormal, inf or nan
        if ((b << 1) == 0) {  // +-0 projects to tile 0
            *out = 0;
            return true;
        }
        return project_coord_fp64(v, pp.scale, out);
    }
    const bool neg = (b >> 63) != 0ull;
    const unsigned long long mx = (b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
    unsigned long long q;
    if (!WIDE) {
        const unsigned long long P = mx * (unsigned long long)(unsigned int)pp.s_odd;  // < 2^63 (s_odd < 2^10)
        const int D = pp.d0 - (int)e;                 // v*s = P * 2^-D
        if (D <= 0) return false;                     // |v*s| >= 2^52
        const int t = pp.top + (int)((P >> pp.top) != 0ull);  // bit length of P
        if (D > t) {                                  // |v*s| < 1/2
            if (D > t + 1021) return project_coord_fp64(v, pp.scale, out);  // subnormal product
            q = neg ? 1ull : 0ull;
        } else {
            const int r = t - 53;                     // 0..10
            const unsigned long long half = (r > 0) ? (1ull << (r - 1)) : 0ull;
            const unsigned long long bias = neg ? ((1ull << D) - 1ull - half) : half;
            q = (P + bias) >> D;                      // D <= t <= 63: no overflow
        }
    } else {
        const unsigned long long lo = mx * pp.s_odd;
        const unsigned long long hi = __umul64hi(mx, pp.s_odd);
        const int t = pp.top + (int)((hi >> (pp.top - 64)) != 0ull);  // 64 <= top <= 105
        const int r = t - 53;                                           // 11..53
        // M = P rounded to 53 significant bits (ties to even), as M * 2^r
        unsigned long long M = (hi << (64 - r)) | (lo >> r);
        const unsigned long long rb = (lo >> (r - 1)) & 1ull;
        const unsigned long long sticky = (lo & ((1ull << (r - 1)) - 1ull)) != 0ull;
        M += rb & (sticky | (M & 1ull));
        const int kk = (int)e - 1075 + pp.s_exp + r;  // RN(v*s) = M * 2^kk
        if (kk < -1074) return project_coord_fp64(v, pp.scale, out);
        const int D = -kk;
        if (D <= 0) return false;
        if (D >= 64) {
            q = neg ? 1ull : 0ull;
        } else {
            const unsigned long long ip = M >> D;
            const unsigned long long fr = (M << (64 - D)) != 0ull;
            q = neg ? ip + fr : ip;
        }
    }
    if (neg) {
        if (q > 2147483647ull) return false;
        *out = -(int)q;
    } else {
        if (q > 2147483646ull) return false;
        *out = (int)q;
    }
    return true;
}

}  // namespace raster
