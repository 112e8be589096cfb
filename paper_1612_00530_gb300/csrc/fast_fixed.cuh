// Fixed-point helpers of the FAST summation order, shared by the kernels
// that compute it (k_spmv.cu, k_tma.cu) so that every kernel rounds the
// same exact integer sum the same way.  Included inside each file's
// anonymous namespace: every translation unit keeps its own internal copy.
//
// FAST order (pattern format, value tables whose entries are small integer
// multiples m of one power of two 2^mult_exp): x_j becomes the 53-bit fixed
// point X_j = sign(x_j) floor(|x_j| 2^(1075 - E)), E a biased exponent at
// least that of every x_j in play, held as two signed limbs
// X = xh 2^26 + xl; a row's sum of m_j X_j is exact in 64-bit integers and
// rounded once to binary64 (scaled by 2^(E - 1075 + mult_exp)).
#pragma once

__device__ __forceinline__ void raise_error(int32_t* err, int32_t code) {
    if (err) atomicOr(err, code);
}

// PTX prmt in its default mode: for each result byte a 4-bit selector picks
// one of the 8 source bytes; a set selector msb replicates that byte's sign.
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// Signed multiplier of value code c (< 8) from the packed int8 table.
__device__ __forceinline__ int32_t mult_of(uint32_t lo, uint32_t hi, uint32_t c) {
    return int32_t(prmt(lo, hi, (c & 7u) * 0x1111u + 0x8880u));
}

__device__ __forceinline__ uint32_t byte_of(const uint32_t (&w)[kMaxRecordWords], int u) {
    return (w[u >> 2] >> (8 * (u & 3))) & 0xFFu;
}

// Row record of the pattern format: `WORDS` 32-bit words split over up to
// three planes indexed by row, so each warp load is one contiguous run.
template <int WORDS>
__device__ __forceinline__ void load_record(const PatternView& a, int64_t r, uint32_t (&w)[kMaxRecordWords]) {
    constexpr int q16 = WORDS / 4, rem = WORDS % 4;
    if (q16 >= 1) {
        const uint4 v = __ldcs(a.p16a + r);
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    }
    if (q16 >= 2) {
        const uint4 v = __ldcs(a.p16b + r);
        w[4] = v.x; w[5] = v.y; w[6] = v.z; w[7] = v.w;
    }
    if (rem >= 2) {
        const uint2 v = __ldcs(a.p8 + r);
        w[4 * q16] = v.x; w[4 * q16 + 1] = v.y;
    }
    if (rem & 1) w[WORDS - 1] = __ldcs(a.p4 + r);
}

// x -> X = sign(x) * floor(|x| * 2^(1075 - E)) as two limbs X = xh*2^26 + xl
// (both carrying the sign), integer operations only.
__device__ __forceinline__ void to_fixed(double xv, int emax, int32_t& xh, int32_t& xl) {
    const uint32_t hi = uint32_t(__double2hiint(xv)), lo = uint32_t(__double2loint(xv));
    const uint32_t k = uint32_t(emax) - ((hi >> 20) & 0x7FFu);
    const uint64_t mant = (uint64_t((hi & 0xFFFFFu) | 0x100000u) << 32) | lo;
    uint64_t X;
    asm("shr.b64 %0, %1, %2;" : "=l"(X) : "l"(mant), "r"(k));  // shifts >= 64 give 0
    const int32_t sgn = int32_t(hi) >> 31;
    xl = (int32_t(uint32_t(X) & 0x3FFFFFFu) ^ sgn) - sgn;
    xh = (int32_t(X >> 26) ^ sgn) - sgn;
}

// acc * 2^S rounded to nearest-even, integer operations only (subnormal
// results are rounded to their shorter precision, overflow gives +-inf).
__device__ __noinline__ double fixed_to_double_int(int64_t acc, int S) {
    if (acc == 0) return 0.0;
    const uint64_t sgn = acc < 0 ? 0x8000000000000000ull : 0ull;
    uint64_t a = acc < 0 ? uint64_t(0) - uint64_t(acc) : uint64_t(acc);
    const int lz = __clzll(a);
    a <<= lz;                                   // leading one at bit 63
    const int e = 63 - lz + S + 1023;           // biased exponent if normal
    // bits of `a` below the kept mantissa: 11 for a normal result, more for a
    // subnormal one (the field then holds the value / 2^-1074 directly)
    const int drop = e >= 1 ? 11 : 12 - e;
    uint64_t mant, rest;
    if (drop >= 65) { mant = 0; rest = 0; }             // below half the smallest subnormal
    else if (drop == 64) { mant = 0; rest = a; }
    else { mant = a >> drop; rest = a << (64 - drop); }
    const uint64_t half = 0x8000000000000000ull;
    mant += (rest > half || (rest == half && (mant & 1u))) ? 1u : 0u;
    uint64_t bits;
    if (e >= 1) {
        // mant in [2^52, 2^53]; a carry to 2^53 moves into the exponent field
        bits = (uint64_t(e - 1) << 52) + mant;
        if (e - 1 + int(mant >> 52) >= 2047) bits = 0x7FF0000000000000ull;
    } else {
        bits = mant;  // subnormal; a carry to 2^52 becomes the smallest normal
    }
    return __longlong_as_double(int64_t(sgn | bits));
}

// acc * 2^S rounded to nearest-even.  The int64 -> binary64 conversion
// rounds once (RN); scaling by 2^S is then an exact add to the exponent
// field unless the result leaves the normal range, which the integer
// routine above handles.  The add is made on the whole 64-bit pattern
// (unsigned, since a negative S shifted left is undefined in C++17): a
// version that added S << 20 to the high word and re-paired it with the
// low word returned the low word replaced by S in the staged kernel at
// eight rows a thread under a 40-register budget (every row after a
// thread's first), although that source has no undefined behaviour.
__device__ __forceinline__ double fixed_to_double(int64_t acc, int S) {
    const double d = __ll2double_rn(acc);
    const uint64_t bits = uint64_t(__double_as_longlong(d));
    const int ef = int(bits >> 52) & 0x7FF;      // 0 exactly when acc == 0
    if (ef != 0 && uint32_t(ef + S - 1) < 2046u)
        return __longlong_as_double(int64_t(bits + (uint64_t(int64_t(S)) << 52)));
    return ef == 0 ? d : fixed_to_double_int(acc, S);
}

// (lo, hi) words of x -> limbs (xl, xh) of X = sign(x) floor(|x| 2^(1075-E)),
// X = xh 2^26 + xl with both limbs carrying the sign.
__device__ __forceinline__ int2 fixed_limbs(uint32_t lo, uint32_t hi, uint32_t emax) {
    const uint32_t k = emax - ((hi >> 20) & 0x7FFu);
    const uint32_t mh = (hi & 0xFFFFFu) | 0x100000u;
    uint64_t X;
    asm("shr.b64 %0, %1, %2;" : "=l"(X) : "l"((uint64_t(mh) << 32) | lo), "r"(k));
    const int32_t s1 = (int32_t(hi) >> 31) | 1;  // +1 or -1
    return make_int2(int32_t(uint32_t(X) & 0x3FFFFFFu) * s1, int32_t(uint32_t(X >> 26)) * s1);
}
