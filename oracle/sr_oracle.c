/*
 * CPU oracle for the device-wide sum reduction — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm may load this library.  The CUDA product path never links it, and it
 * shares no header, helper or constant with the CUDA sources.
 *
 * What it computes is the plain definition of the case-study operator of the
 * paper ("Case Study: Reduction Operator", Section VII): the sum of the
 * elements of an array, S = sum_{i<n} x_i.  Every routine below is that
 * definition written out as a sequential loop, in the widest arithmetic that
 * keeps it obviously correct:
 *
 *   - int32 input: an int64 loop (exact for n <= 2^32, since |x_i| <= 2^31).
 *   - floating-point input: an FP64 loop over the decoded values (carries its
 *     own rounding error, at most (n-1) * 2^-53 * sum|x_i|), and an EXACT
 *     fixed-point (Kulisch-style) accumulator.  Every finite binary32 value is
 *     an integer multiple of 2^-149 below 2^128, so a wide two's-complement
 *     integer held in 32-bit digits stored in int64 limbs sums any number of
 *     them without rounding.  The caller rounds the digits once (Python's
 *     int / int division is correctly rounded).
 *   - BF16 input: the 16 stored bits are the top half of a binary32 word, so
 *     decoding is a 16-bit left shift (exact).
 *   - FP8 E4M3 input: decoded from its bit fields (1 sign, 4 exponent bits
 *     with bias 7, 3 mantissa bits; exponent 0 is subnormal, code S.1111.111
 *     is NaN, there is no infinity; largest finite magnitude 448).  The
 *     per-tensor dequantisation scale is a factor of the whole sum, so the
 *     FP64 routine multiplies each decoded value by it and the exact routine
 *     sums the unscaled codes (the caller multiplies by the scale exactly).
 *   - segmented input (CSR offsets): the same loops, once per segment.
 *
 * Non-finite inputs are outside the oracle's domain: the exact routines stop
 * and return -1 when they meet one.
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

/* Number of 32-bit digits in the exact accumulator.  Bit k of the fixed-point
 * integer has weight 2^(k-149).  A binary32 magnitude is below 2^24 * 2^253
 * (bit 277), the sum of up to 2^33 terms adds 33 bits, and one more digit
 * holds the sign: 12 digits = 384 bits is ample. */
#define ORACLE_LIMBS 12

int oracle_limbs(void) { return ORACLE_LIMBS; }

/* ---------------------------------------------------------------- int32 */

int64_t oracle_sum_i32(const int32_t* x, int64_t n) {
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i) s += (int64_t)x[i];
    return s;
}

/* ----------------------------------------------------------- decoding */

static float bf16_to_f32(uint16_t b) {
    uint32_t w = ((uint32_t)b) << 16;
    float f;
    memcpy(&f, &w, sizeof f);
    return f;
}

/* FP8 E4M3 (OCP "E4M3FN" layout) decoded to its exact value. */
static double e4m3_to_f64(uint8_t c) {
    int sign = (c >> 7) & 1;
    int e = (c >> 3) & 0xF;
    int m = c & 0x7;
    double v;
    if (e == 0xF && m == 0x7) return NAN;
    if (e == 0)
        v = ldexp((double)m, -9);              /* (m/8) * 2^(1-7) */
    else
        v = ldexp((double)(8 + m), e - 10);    /* (1 + m/8) * 2^(e-7) */
    return sign ? -v : v;
}

double oracle_decode_e4m3(uint8_t c) { return e4m3_to_f64(c); }
double oracle_decode_bf16(uint16_t b) { return (double)bf16_to_f32(b); }

/* ------------------------------------------------------- FP64 loops */

double oracle_sum_f32(const float* x, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += (double)x[i];
    return s;
}

double oracle_sum_bf16(const uint16_t* x, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += (double)bf16_to_f32(x[i]);
    return s;
}

double oracle_sum_e4m3(const uint8_t* q, int64_t n, double scale) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += e4m3_to_f64(q[i]) * scale;
    return s;
}

/* sum of |x_i| in FP64 (used only to state error bounds) */
double oracle_sum_abs_f32(const float* x, int64_t n) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += fabs((double)x[i]);
    return s;
}

/* ----------------------------------------------- exact accumulator */

/* Carry-propagate: digit k keeps bits [32k, 32k+32) in [0, 2^32), the top
 * digit keeps the sign.  Arithmetic right shift of a negative int64 is
 * implementation-defined in C, so the borrow is computed explicitly. */
static void limbs_normalise(int64_t* L) {
    for (int k = 0; k < ORACLE_LIMBS - 1; ++k) {
        int64_t v = L[k];
        int64_t low = (int64_t)((uint64_t)v & 0xFFFFFFFFull);
        int64_t carry = (v - low) / 4294967296LL;   /* exact division */
        L[k] = low;
        L[k + 1] += carry;
    }
}

/* Add sign * mant * 2^(shift - 149) with 0 <= mant < 2^25, 0 <= shift. */
static void limbs_add(int64_t* L, int sign, uint64_t mant, int shift) {
    int k = shift / 32, off = shift % 32;
    uint64_t wide = mant << off;                  /* < 2^57 */
    int64_t lo = (int64_t)(wide & 0xFFFFFFFFull);
    int64_t hi = (int64_t)(wide >> 32);
    if (sign) { lo = -lo; hi = -hi; }
    L[k] += lo;
    L[k + 1] += hi;
}

/* Decompose a finite binary32 into (sign, integer mantissa, shift) so that
 * value = (-1)^sign * mant * 2^(shift-149). Returns 0 for finite, -1 else. */
static int f32_fields(float f, int* sign, uint64_t* mant, int* shift) {
    uint32_t w;
    memcpy(&w, &f, sizeof w);
    uint32_t eb = (w >> 23) & 0xFF, frac = w & 0x7FFFFF;
    if (eb == 0xFF) return -1;
    *sign = (int)(w >> 31);
    if (eb == 0) { *mant = frac; *shift = 0; }
    else { *mant = (uint64_t)frac | 0x800000u; *shift = (int)eb - 1; }
    return 0;
}

#define ORACLE_RENORM_EVERY (1LL << 26)

int oracle_exact_f32(const float* x, int64_t n, int64_t* L) {
    memset(L, 0, sizeof(int64_t) * ORACLE_LIMBS);
    for (int64_t i = 0; i < n; ++i) {
        int sg, sh; uint64_t m;
        if (f32_fields(x[i], &sg, &m, &sh)) return -1;
        limbs_add(L, sg, m, sh);
        if ((i + 1) % ORACLE_RENORM_EVERY == 0) limbs_normalise(L);
    }
    limbs_normalise(L);
    return 0;
}

int oracle_exact_bf16(const uint16_t* x, int64_t n, int64_t* L) {
    memset(L, 0, sizeof(int64_t) * ORACLE_LIMBS);
    for (int64_t i = 0; i < n; ++i) {
        int sg, sh; uint64_t m;
        if (f32_fields(bf16_to_f32(x[i]), &sg, &m, &sh)) return -1;
        limbs_add(L, sg, m, sh);
        if ((i + 1) % ORACLE_RENORM_EVERY == 0) limbs_normalise(L);
    }
    limbs_normalise(L);
    return 0;
}

/* Exact sum of the UNSCALED decoded E4M3 values; each is a multiple of 2^-9,
 * so it is added as an integer count of 2^-9 (= 2^140 * 2^-149). */
int oracle_exact_e4m3(const uint8_t* q, int64_t n, int64_t* L) {
    memset(L, 0, sizeof(int64_t) * ORACLE_LIMBS);
    for (int64_t i = 0; i < n; ++i) {
        uint8_t c = q[i];
        int e = (c >> 3) & 0xF, m = c & 0x7;
        if (e == 0xF && m == 0x7) return -1;
        uint64_t units = (e == 0) ? (uint64_t)m : ((uint64_t)(8 + m) << (e - 1));
        limbs_add(L, (c >> 7) & 1, units, 140);
        if ((i + 1) % ORACLE_RENORM_EVERY == 0) limbs_normalise(L);
    }
    limbs_normalise(L);
    return 0;
}

/* ------------------------------------------------------ segmented */

/* out[s] = sum of x[offsets[s] .. offsets[s+1]) ; offsets has nseg+1 entries */
void oracle_segsum_f32(const float* x, const int64_t* offsets, int64_t nseg,
                       double* out) {
    for (int64_t s = 0; s < nseg; ++s) {
        double acc = 0.0;
        for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) acc += (double)x[i];
        out[s] = acc;
    }
}

void oracle_segsum_i32(const int32_t* x, const int64_t* offsets, int64_t nseg,
                       int64_t* out) {
    for (int64_t s = 0; s < nseg; ++s) {
        int64_t acc = 0;
        for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) acc += (int64_t)x[i];
        out[s] = acc;
    }
}

/* exact per-segment sums: out_limbs is nseg * ORACLE_LIMBS int64 */
int oracle_segexact_f32(const float* x, const int64_t* offsets, int64_t nseg,
                        int64_t* out_limbs) {
    for (int64_t s = 0; s < nseg; ++s) {
        int64_t* L = out_limbs + s * ORACLE_LIMBS;
        if (oracle_exact_f32(x + offsets[s], offsets[s + 1] - offsets[s], L))
            return -1;
    }
    return 0;
}

void oracle_segsum_abs_f32(const float* x, const int64_t* offsets, int64_t nseg,
                           double* out) {
    for (int64_t s = 0; s < nseg; ++s) {
        double acc = 0.0;
        for (int64_t i = offsets[s]; i < offsets[s + 1]; ++i) acc += fabs((double)x[i]);
        out[s] = acc;
    }
}
