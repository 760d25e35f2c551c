// bls_kernels.cu -- sm_103a kernels of the box-least-squares search (Sec. 2.2.2).
//
//  prep_kernel        one block per curve: weights, weighted mean, mean-subtracted flux,
//                     time offsets (FP64), stored as 16-byte points for the hot loop.
//  fold_sweep_kernel  persistent; one work item = (curve, tile of T frequencies); one
//                     thread per frequency with a private phase histogram in shared
//                     memory.  Loop A folds and bins every point; loop B sweeps every
//                     cyclic box and keeps the largest power P of the frequency.
//  reduce_kernel      one block per curve: top-k peaks of P over frequencies, the best box
//                     (i1, k) of each peak frequency with the exact tie-break, FP64 refit of
//                     that box, reported quantities.
//  argmax_kernel      the best box of listed frequencies (diagnostics).
//  plain_f64_kernel   baseline, one curve per launch, one thread per frequency, FP64
//                     histograms in global memory (the paper's decomposition).
//
// Fold semantics (identical to the FP64 definition): p = RN(dt*f), phase = p - floor(p),
// bin = floor(RN(phase*nb)) clamped to nb-1.  The fast path evaluates dt*f as a
// double-FP32 product with a proven error bound and re-folds in FP64 only the points that
// lie within that bound of a bin edge, so every bin equals the FP64 one.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "bls.h"
#include "bls_internal.h"

namespace blsgpu {

// ------------------------------------------------------------------------- fold

__device__ __forceinline__ double grid_freq(const CurveDesc& cd, int j)
{
    if (cd.freqs) return cd.freqs[j];
    return __dadd_rn(cd.fmin, __dmul_rn((double)j, cd.df));
}

// Exact fold in FP64, every operation rounded once (no contraction).
__device__ __forceinline__ unsigned fold_exact(double dt, double f, int nb)
{
    double p = __dmul_rn(dt, f);
    double ph = __dsub_rn(p, floor(p));
    double u = __dmul_rn(ph, (double)nb);
    int b = (int)floor(u);
    b = b >= nb ? nb - 1 : b;
    return (unsigned)(b < 0 ? 0 : b);
}

// Constants of the fold of one thread's frequency.
struct FoldConst {
    float fh, fl;     // f = fh + fl (+ |err| <= 2^-48 f)
    float nbf;        // nb as float
    float lim;        // 0.5 - tol: |d| beyond this means "near a bin edge"
    double f;         // exact frequency
    int nb;
    bool fast;        // the double-FP32 path is valid for this (curve, frequency)
    // fixed-point fold (FX64)
    unsigned Flo, Fhi;   // F = RN_int(f 2^(64 - fxs))
    unsigned ftol;       // edge window: bin certain iff ftol <= r < 2^32 - ftol - nb
    unsigned fspan;      // 2^32 - 2 ftol - nb
    bool fxok;           // the fixed-point path is valid for this (curve, frequency)
    // incremental fixed-point fold of a uniform-grid tile (see make_fold_const_inc)
    unsigned tau;        // j - jc (two's complement): this column's offset from the reference
    unsigned Fclo, Fchi; // Fc = RN_int(f_jc 2^(64 - fxs))
    unsigned dFlo, dFhi; // dF = RN_int(df 2^(96 - fxs)) < 2^63
    unsigned sh;         // log2 nb when nb is a power of two (the bin is then a shift)
};

// Fixed-point scale of a curve's offsets: DT = RN_int(dt 2^s) with dt < 2^L.  The fold
// error f 2^-(s+1) + dtmax 2^(s-65) (see make_fold_const) is smallest near
// s = 32 + (log2 f - L) / 2; s = 34 - (L+1)/2 suits frequencies up to ~16 cycles per unit
// of time, and DT < 2^62 leaves headroom.
__host__ __device__ __forceinline__ int fx_shift(double dtmax)
{
    int L = 0;
    if (dtmax > 0.0) L = ilogb(dtmax) + 1;
    int s = 34 - (L + 1) / 2;
    if (s > 62 - L) s = 62 - L;
    return s < 1 ? 1 : s;
}

// 2^e as an FP64 number built from its exponent field, for -1022 <= e <= 1023: x * pow2(e)
// equals ldexp(x, e) whenever the result is a normal number (every use below), at the cost
// of one FP64 multiply.
__device__ __forceinline__ double pow2(int e)
{
    return __hiloint2double((e + 1023) << 20, 0);
}

// Error bound of the double-FP32 fold, in bins.  With D = dt, F = f, DF = D*F and
// u = 2^-24 (FP32 unit roundoff):
//   split errors |D - dh - dl| <= u^2 D, |F - fh - fl| <= u^2 F, dropped dl*fl <= u^2 DF,
//   two-product exact, two FMA roundings of the cross terms <= 1.5 u^2 DF
//   => |ph + c - DF| <= 2^-44 DF cycles;
//   cn = RN(c nb - 1/2) and x = RN(fr nb + cn) add u|cn| + u|x|;
//   the FP64 definition itself is within nb 2^-53 (DF + 1) bins of nb*frac(DF).
// tol doubles the sum.  Valid while DF < 2^20 (then |c| < 3u DF < 0.19 cycles).
//
// Fixed-point fold (FX64), with s = fxs: the prep kernel stores DT = RN_int(dt 2^s) and
// F = RN_int(f 2^(64-s)), so |DT F 2^-64 - dt f| <= f 2^-(s+1) + dt 2^(s-65) + 2^-66 =: E
// cycles, and the low 64 bits of DT*F are the phase frac(dt f) in units of 2^-64 up to E.
// Only the high word q of that fraction is formed; b = floor(q nb 2^-32), r = q nb mod
// 2^32, and the dropped low word adds less than nb to r.  The FP64 definition lies within
// 2^-52 (DF + 1) nb bins of nb*frac(dt f), so b is the definition's bin whenever r is at
// least tol = (E + 2^-52 (DF + 1)) nb 2^32 (with margin) from both ends of the bin:
// tol <= r < 2^32 - tol - nb.
//
// The hot kernels ask only for the parts their fold uses: `direct` (the FX64 constants of
// the direct fold; a tile on the incremental fold sets its own) and `df32` (the double-FP32
// and FP32 folds' constants); the per-tile constants are FP64 arithmetic, a slow pipe on
// this GPU.
__device__ __forceinline__ FoldConst make_fold_const(double f, int nb, double dtmax, int fxs,
                                                     bool direct = true, bool df32 = true)
{
    FoldConst fc;
    fc.fxok = false;
    fc.Flo = fc.Fhi = fc.ftol = fc.fspan = 0u;
    if (direct) {
        const double Fd = f * pow2(64 - fxs);
        fc.fxok = Fd < 18446744073709551616.0;   // F < 2^64
        const unsigned long long F = fc.fxok ? __double2ull_rn(Fd) : 0ull;
        fc.Flo = (unsigned)F;
        fc.Fhi = (unsigned)(F >> 32);
        const double E = f * pow2(-(fxs + 1)) + dtmax * pow2(fxs - 65) + pow2(-66)
                       + pow2(-52) * (dtmax * f + 1.0);
        const double tolu = E * nb * 4294967296.0 * 1.01 + 4.0;
        fc.fxok = fc.fxok && tolu < 1.0e9;
        const unsigned tol = fc.fxok ? (unsigned)ceil(tolu) : 0u;
        fc.ftol = tol;
        fc.fspan = fc.fxok ? (unsigned)(4294967296.0 - 2.0 * tol - nb) : 0u;
    }
    fc.f = f;
    fc.nb = nb;
    fc.sh = (nb & (nb - 1)) == 0 ? 31u - (unsigned)__clz(nb) : 0u;
    fc.nbf = (float)nb;
    fc.fh = fc.fl = 0.0f;
    fc.fast = false;
    fc.lim = 0.0f;
    if (!df32) return fc;
    fc.fh = __double2float_rn(f);
    fc.fl = __double2float_rn(__dsub_rn(f, (double)fc.fh));
    double DF = dtmax * f;
    fc.fast = DF < 1048576.0;
    double cmax = 3.0 * 5.9604644775390625e-8 * DF;          // 3 u DF
    double cn = cmax * nb + 0.5;
    double xm = nb * (0.5 + cmax) + 0.5 + cn;
    double tol = 2.0 * (nb * DF * 5.684341886080802e-14       // 2^-44
                        + 5.9604644775390625e-8 * (cn + xm)    // u (|cn| + |x|)
                        + nb * 2.220446049250313e-16 * (DF + 1.0));  // 2^-52
    fc.lim = __double2float_rd(0.5 - tol);
    return fc;
}

// Incremental fixed-point fold of a uniform-grid tile.  The tile's columns j share one
// reference column jc; per point, the tile's staging step forms once
//   Qi = the FX64 phase word of dt_i at f_jc   (floor(DT Fc 2^-32) mod 2^32, as above),
//   Di = RN(DT dF 2^-64) mod 2^32               (the phase step frac(dt_i df) in 2^-32 units),
// and the column with offset tau = j - jc takes q = Qi + tau Di (mod 2^32): one integer
// multiply-add per point and frequency instead of three.  Relative to dt f_j (mod 1), with
// f_j = RN(fmin + RN(j df)):
//   Qi 2^-32 lies in (X - 2^-32, X] with |X - dt f_jc| <= f_jc 2^-(s+1) + dtmax 2^(s-65) + 2^-66,
//   |Di 2^-32 - dt df| <= 2^-33 + df 2^-(s+1) + dtmax 2^(s-97) + 2^-98 (multiplied by |tau|),
//   |dt f_j - dt (f_jc + tau df)| <= dtmax fmax 2^-51 (1.01) (both grid roundings),
// and the FP64 definition is within 2^-52 (dt f_j + 1) of dt f_j, so the window test of the
// direct fold applies with tol = (sum of these) nb 2^32 (1.01) + 4.  Valid (fxok) while
// Fc < 2^64, dF < 2^63 and tol < 10^9; the window keeps fewer than 10^-5 of the points of
// the typical workloads for the exact re-fold.
__device__ __forceinline__ bool inc_tile_ok(double fcen, const CurveDesc& cd)
{
    return cd.incok && fcen >= 0.0 && fcen * pow2(64 - cd.fxs) < 18446744073709551616.0;
}

// The per-curve terms (dF, the coefficients of E) come from the prep kernel; a tile computes
// Fc in FP64 and its columns' windows in FP32 with every operation rounded up, so the window
// is never narrower than the bound (and the FP64 pipe, slow on this GPU, does little).
__device__ __forceinline__ void make_fold_const_inc(FoldConst& fc, double f, double fcen, int tau,
                                                    const CurveDesc& cd, int nb)
{
    const unsigned long long Fc = __double2ull_rn(fcen * pow2(64 - cd.fxs));
    fc.Fclo = (unsigned)Fc;
    fc.Fchi = (unsigned)(Fc >> 32);
    fc.dFlo = (unsigned)cd.dF;
    fc.dFhi = (unsigned)(cd.dF >> 32);
    fc.tau = (unsigned)tau;
    const float ff = __double2float_ru(f), fcf = __double2float_ru(fcen);
    const float at = (float)(tau < 0 ? -tau : tau);   // exact: |tau| < 2^24
    float E = __fmaf_ru(fcf, cd.ewc, cd.ew0);
    E = __fmaf_ru(at, cd.ewt, E);
    E = __fmaf_ru(fmaxf(ff, fcf), cd.ewh, E);
    E = __fmaf_ru(ff, cd.ewf, E);
    // tol = E nb 2^32 (1.01) + 4, rounded up
    const float tolu = __fadd_ru(__fmul_ru(__fmul_ru(__fmul_ru(E, (float)nb), 4294967296.0f), 1.0101f), 4.0f);
    fc.fxok = tolu < 1.0e9f;
    const unsigned tol = fc.fxok ? __float2uint_ru(tolu) : 0u;
    fc.ftol = tol;
    fc.fspan = fc.fxok ? 0u - 2u * tol - (unsigned)nb : 0u;   // 2^32 - 2 tol - nb
}

// (Qi, Di) of one point from DT = (hi:lo) and the tile's Fc, dF (see make_fold_const_inc).
__device__ __forceinline__ void inc_point(unsigned lo, unsigned hi, const FoldConst& fc,
                                          unsigned& Q, unsigned& D)
{
    Q = __umulhi(lo, fc.Fclo) + lo * fc.Fchi + hi * fc.Fclo;
    // bits 64..95 of DT dF rounded to nearest: DT dF = p00 + 2^32 (p01 + p10) + 2^64 hi dFhi
    typedef unsigned long long w64;
    const w64 p00 = (w64)lo * fc.dFlo, p01 = (w64)lo * fc.dFhi, p10 = (w64)hi * fc.dFlo;
    const w64 mid = (p00 >> 32) + (w64)(unsigned)p01 + (w64)(unsigned)p10 + 0x80000000ull;
    D = (unsigned)(mid >> 32) + (unsigned)(p01 >> 32) + (unsigned)(p10 >> 32) + hi * fc.dFhi;
}

// Staging step of the incremental fold on the copies this thread made of a chunk (slots
// i = tid + m*nthreads < cn; nthreads even, so the thread's slots are all point-pair DT
// slots or all weight slots): (lo0, lo1, hi0, hi1) -> (Q0, Q1, D0, D1).  Runs after the
// thread's cp.async copies of the chunk completed and before the barrier that publishes it.
__device__ __forceinline__ void inc_stage(float4* dp, int cn, int tid, int nthreads,
                                          const FoldConst& fc)
{
    if (tid & 1) return;
    for (int i = tid; i < cn; i += nthreads) {
        const float4 A = dp[i];
        unsigned Q0, D0, Q1, D1;
        inc_point(__float_as_uint(A.x), __float_as_uint(A.z), fc, Q0, D0);
        inc_point(__float_as_uint(A.y), __float_as_uint(A.w), fc, Q1, D1);
        dp[i] = make_float4(__uint_as_float(Q0), __uint_as_float(Q1), __uint_as_float(D0),
                            __uint_as_float(D1));
    }
}

// FP32 fold (precision study): no error bound, no fallback.
__device__ __forceinline__ unsigned fold_f32(float dt32, const FoldConst& fc)
{
    float p = __fmul_rn(dt32, fc.fh);
    float ph = __fsub_rn(p, floorf(p));
    int b = (int)floorf(__fmul_rn(ph, fc.nbf));
    b = b >= fc.nb ? fc.nb - 1 : b;
    return (unsigned)(b < 0 ? 0 : b);
}

// ---- packed FP32 pairs (f32x2: one instruction, two lanes of FP32 arithmetic)
typedef unsigned long long u64;

__device__ __forceinline__ u64 pk(float lo, float hi)
{
    u64 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(u64 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
#ifdef BLS_SCALAR_PAIRS
// Pair arithmetic spelled as two scalar FP32 instructions (same rounding, per lane).
__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    float a0, a1, b0, b1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    return pk(__fadd_rn(a0, b0), __fadd_rn(a1, b1));
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    float a0, a1, b0, b1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    return pk(__fsub_rn(a0, b0), __fsub_rn(a1, b1));
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    float a0, a1, b0, b1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    return pk(__fmul_rn(a0, b0), __fmul_rn(a1, b1));
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    float a0, a1, b0, b1, c0, c1;
    upk(a, a0, a1);
    upk(b, b0, b1);
    upk(c, c0, c1);
    return pk(__fmaf_rn(a0, b0, c0), __fmaf_rn(a1, b1, c1));
}
// acc + x where i == j, else acc.
__device__ __forceinline__ u64 add2_if_eq(u64 acc, u64 x, unsigned i, unsigned j)
{
    return i == j ? add2(acc, x) : acc;
}
#else
__device__ __forceinline__ u64 add2(u64 a, u64 b)
{
    u64 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b)
{
    u64 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b)
{
    u64 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c)
{
    u64 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// acc + x where i == j, else acc: one compare and one predicated packed add.
__device__ __forceinline__ u64 add2_if_eq(u64 acc, u64 x, unsigned i, unsigned j)
{
    asm("{\n\t.reg .pred p;\n\tsetp.eq.u32 p, %2, %3;\n\t@p add.rn.f32x2 %0, %0, %1;\n\t}"
        : "+l"(acc) : "l"(x), "r"(i), "r"(j));
    return acc;
}

#endif

// Constants of the double-FP32 fold as broadcast pairs.
struct FoldPacked {
    u64 FH, NFH, FL, M, NB, NNB, MHALF;
    float lim;
    int nb;
};

__device__ __forceinline__ FoldPacked make_fold_packed(const FoldConst& fc)
{
    FoldPacked q;
    const float M = 12582912.0f;
    q.FH = pk(fc.fh, fc.fh);
    q.NFH = pk(-fc.fh, -fc.fh);
    q.FL = pk(fc.fl, fc.fl);
    q.M = pk(M, M);
    q.NB = pk(fc.nbf, fc.nbf);
    q.NNB = pk(-fc.nbf, -fc.nbf);
    q.MHALF = pk(-0.5f, -0.5f);
    q.lim = fc.lim;
    q.nb = fc.nb;
    return q;
}

// Double-FP32 fold of two points at once.  With dt = dh + dl and f = fh + fl:
//   ph = RN(dh fh) and e = dh fh - ph (exact, by FMA) give the product's high part,
//   c = dl fh + dh fl + e its low part, so dt f ~= ph + c (error <= 2^-44 dt f);
//   fr = ph - rint(ph) (exact, in [-1/2, 1/2]) is the phase mod 1, centred;
//   x = fr nb + c nb - 1/2, and rint(x) = floor(nb phase) up to a multiple of nb;
//   d = x - rint(x): when |d| <= lim the bin is certain, otherwise (edge) it is re-folded
//   in FP64.  rint uses RN(v + 1.5 2^23) - 1.5 2^23, valid for |v| < 2^22.
// Packed instructions have no negation modifier, so ph and fr are carried negated.
__device__ __forceinline__ void fold_df32_pair(const float4& A, const FoldPacked& q,
                                               unsigned& b0, unsigned& b1, bool& e0, bool& e1)
{
    const u64 DH = pk(A.x, A.y), DL = pk(A.z, A.w);
    const u64 NPH = mul2(DH, q.NFH);
    const u64 E = fma2(DH, q.FH, NPH);
    const u64 T1 = fma2(DH, q.FL, E);
    const u64 C = fma2(DL, q.FH, T1);
    const u64 MM = add2(NPH, q.M);
    const u64 NRP = sub2(MM, q.M);
    const u64 NFR = sub2(NPH, NRP);
    const u64 CN = fma2(C, q.NB, q.MHALF);
    const u64 X = fma2(NFR, q.NNB, CN);
    const u64 M2 = add2(X, q.M);
    const u64 RX = sub2(M2, q.M);
    const u64 D = sub2(X, RX);
    float d0, d1, m0, m1;
    upk(D, d0, d1);
    upk(M2, m0, m1);
    const int Mb = __float_as_int(12582912.0f);
    const unsigned r0 = (unsigned)(__float_as_int(m0) - Mb), r1 = (unsigned)(__float_as_int(m1) - Mb);
    b0 = min(r0, r0 + (unsigned)q.nb);
    b1 = min(r1, r1 + (unsigned)q.nb);
    e0 = !(fabsf(d0) <= q.lim);   // NaN (bad input) also takes the exact path
    e1 = !(fabsf(d1) <= q.lim);
}

// Fixed-point fold of two points at once.  Direct (INC = false): A = (DT0 lo, DT1 lo, DT0 hi,
// DT1 hi) as bit patterns; the high word of the low 64 bits of DT*F is lo*Fhi + hi*Flo +
// the carry word of lo*Flo (mod 2^32): three integer multiply-adds per point.  Incremental
// (INC = true, a uniform-grid tile after its staging step): A = (Q0, Q1, D0, D1) and the
// phase word is Q + tau D, one multiply-add.  Then one multiply-add for the bin.
template <bool INC = false, bool POW2 = false>
__device__ __forceinline__ void fold_fx_pair(const float4& A, const FoldConst& fc,
                                             unsigned& b0, unsigned& b1, bool& e0, bool& e1)
{
    const unsigned lo0 = __float_as_uint(A.x), lo1 = __float_as_uint(A.y);
    const unsigned hi0 = __float_as_uint(A.z), hi1 = __float_as_uint(A.w);
    unsigned q0, q1;
    if (INC) {
        q0 = lo0 + hi0 * fc.tau;
        q1 = lo1 + hi1 * fc.tau;
    } else {
        q0 = __umulhi(lo0, fc.Flo) + lo0 * fc.Fhi + hi0 * fc.Flo;
        q1 = __umulhi(lo1, fc.Flo) + lo1 * fc.Fhi + hi1 * fc.Flo;
    }
    const unsigned nbu = (unsigned)fc.nb;
    if (POW2) {   // nb = 2^sh: bin and in-bin place are the phase word's top and low bits
        b0 = q0 >> (32u - fc.sh);
        b1 = q1 >> (32u - fc.sh);
        e0 = q0 * nbu - fc.ftol >= fc.fspan;   // q nb = q << sh: one multiply-add
        e1 = q1 * nbu - fc.ftol >= fc.fspan;
    } else {
        b0 = __umulhi(q0, nbu);
        b1 = __umulhi(q1, nbu);
        e0 = q0 * nbu - fc.ftol >= fc.fspan;
        e1 = q1 * nbu - fc.ftol >= fc.fspan;
    }
}

// Fold of the point pair (2p, 2p+1) in a given phase mode; A = (dh0, dh1, dl0, dl1), or
// the fixed-point offsets in FX64 mode.
template <int PHASE>
__device__ __forceinline__ void fold_pair(const float4& A, const double* dtp, const FoldConst& fc,
                                          const FoldPacked& q, unsigned& b0, unsigned& b1)
{
    if (PHASE == kPhaseFX64) {
        bool e0 = true, e1 = true;
        if (fc.fxok) fold_fx_pair(A, fc, b0, b1, e0, e1);
        if (e0) b0 = fold_exact(dtp[0], fc.f, fc.nb);
        if (e1) b1 = fold_exact(dtp[1], fc.f, fc.nb);
    } else if (PHASE == kPhaseF64 || !fc.fast) {
        b0 = fold_exact(dtp[0], fc.f, fc.nb);
        b1 = fold_exact(dtp[1], fc.f, fc.nb);
    } else if (PHASE == kPhaseF32) {
        b0 = fold_f32(__fadd_rn(A.x, A.z), fc);
        b1 = fold_f32(__fadd_rn(A.y, A.w), fc);
    } else {
        bool e0, e1;
        fold_df32_pair(A, q, b0, b1, e0, e1);
        if (e0 | e1) {
            if (e0) b0 = fold_exact(dtp[0], fc.f, fc.nb);
            if (e1) b1 = fold_exact(dtp[1], fc.f, fc.nb);
        }
    }
}

__device__ __forceinline__ void fold_pair_rt(int phase, const float4& A, const double* dtp,
                                             const FoldConst& fc, const FoldPacked& q,
                                             unsigned& b0, unsigned& b1)
{
    if (phase == kPhaseF64) fold_pair<kPhaseF64>(A, dtp, fc, q, b0, b1);
    else if (phase == kPhaseF32) fold_pair<kPhaseF32>(A, dtp, fc, q, b0, b1);
    else if (phase == kPhaseDF32) fold_pair<kPhaseDF32>(A, dtp, fc, q, b0, b1);
    else fold_pair<kPhaseFX64>(A, dtp, fc, q, b0, b1);
}

// ------------------------------------------------------------------------- misc helpers

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}


// Deterministic block sum of FP64 (fixed tree, blockDim.x a power of two <= 1024).
__device__ double block_sum(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = __dadd_rn(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_min(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double* red)
{
    red[threadIdx.x] = v;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

// ------------------------------------------------------------------------- a1: prep

constexpr int kPrepThreads = 256;

// Weights w = dy^-2/W, mean ybar = y0 + sum w (y - y0) (constant flux gives exact zeros),
// x = y - ybar, dt = t - min t.  Points are stored in pairs (2p, 2p+1) as two float4:
// (dt_hi0, dt_hi1, dt_lo0, dt_lo1) and (w0, wx0, w1, wx1), dt in FP64 beside them; an odd
// curve gets a pad point of zero weight.  In the FX64 phase mode the first float4 holds
// the bit patterns of DT = RN_int(dt 2^fxs) instead: (lo0, lo1, hi0, hi1).  In the
// fixed-point sum mode the second float4 holds the bit patterns of the integers
// W = RN(w Sw) (unsigned) and X = RN(w x Sx) (signed) instead of w and w x, with
// Sw = 2^32 - 2n - 16 and Sx = (2^31 - n - 16) / sum |w x|: every subset's W sum is below
// 2^32 and its |X sum| below 2^31, so a bin's integer sums never overflow; the curve's
// wq = 1 / sum W and xq = 1 / Sx turn them back into r and s.  Validates the inputs (finite
// t and y, finite dy > 0, frequencies > 0).
__global__ void __launch_bounds__(kPrepThreads) prep_kernel(CurveDesc* curves, const int* slots,
                                                             int* err, int phase, int sums)
{
    __shared__ double red[kPrepThreads];
    CurveDesc* cd = &curves[slots ? slots[blockIdx.x] : (int)blockIdx.x];
    const int n = cd->n;
    const double* t = cd->t;
    const float* y = cd->y;
    const float* dy = cd->dy;
    float4* pts = cd->pts;
    double* dt64 = cd->dt64;
    bool bad = false;
    double tmin = INFINITY, tmax = -INFINITY, W = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double ti = t[i];
        float yi = y[i];
        if (!isfinite(ti) || !isfinite(yi)) bad = true;
        double inv = 1.0;
        if (dy) {
            float d = dy[i];
            if (!(d > 0.0f) || !isfinite(d)) bad = true;
            double dd = (double)d;
            inv = __ddiv_rn(1.0, __dmul_rn(dd, dd));
        }
        tmin = fmin(tmin, ti);
        tmax = fmax(tmax, ti);
        W = __dadd_rn(W, inv);
    }
    if (cd->freqs) {
        for (int j = threadIdx.x; j < cd->nf; j += blockDim.x) {
            double f = cd->freqs[j];
            if (!(f > 0.0) || !isfinite(f)) bad = true;
        }
    }
    if (bad) atomicOr(err, kErrInput);
    tmin = block_min(tmin, red);
    tmax = block_max(tmax, red);
    W = block_sum(W, red);
    const double y0 = (double)y[0];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double inv = 1.0;
        if (dy) { double dd = (double)dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, W);
        acc = __dadd_rn(acc, __dmul_rn(w, __dsub_rn((double)y[i], y0)));
    }
    acc = block_sum(acc, red);
    const double ybar = __dadd_rn(y0, acc);
    const int fxs = fx_shift(__dsub_rn(tmax, tmin));
    const bool fx = phase == kPhaseFX64;
    const bool fixs = sums == kSumFixed;
    double Sw = 0.0, Sx = 1.0;
    if (fixs) {
        double ax = 0.0;   // sum |w x|
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double inv = 1.0;
            if (dy) { double dd = (double)dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
            const double w = __ddiv_rn(inv, W);
            ax = __dadd_rn(ax, fabs(__dmul_rn(w, __dsub_rn((double)y[i], ybar))));
        }
        ax = block_sum(ax, red);
        Sw = 4294967296.0 - 2.0 * n - 16.0;
        if (ax > 0.0) Sx = __ddiv_rn(2147483648.0 - (double)n - 16.0, ax);
    }
    double swx2 = 0.0, wtot = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double inv = 1.0;
        if (dy) { double dd = (double)dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, W);
        double dt = __dsub_rn(t[i], tmin);
        double x = __dsub_rn((double)y[i], ybar);
        double wx = __dmul_rn(w, x);
        float* A = reinterpret_cast<float*>(&pts[(i >> 1) * 2]);
        float* B = A + 4;
        const int l = i & 1;
        if (fx) {
            const unsigned long long DT = __double2ull_rn(ldexp(dt, fxs));
            A[l] = __uint_as_float((unsigned)DT);
            A[2 + l] = __uint_as_float((unsigned)(DT >> 32));
        } else {
            const float dh = __double2float_rn(dt);
            A[l] = dh;
            A[2 + l] = __double2float_rn(__dsub_rn(dt, (double)dh));
        }
        if (fixs) {
            const unsigned Wi = __double2uint_rn(__dmul_rn(w, Sw));
            B[2 * l] = __uint_as_float(Wi);
            B[2 * l + 1] = __int_as_float(__double2int_rn(__dmul_rn(wx, Sx)));
            wtot = __dadd_rn(wtot, (double)Wi);   // integers below 2^32: exact
        } else {
            B[2 * l] = __double2float_rn(w);
            B[2 * l + 1] = __double2float_rn(wx);
        }
        dt64[i] = dt;
        swx2 = __dadd_rn(swx2, __dmul_rn(wx, x));
    }
    if ((n & 1) && threadIdx.x == 0) {   // pad point of an odd curve: weight 0 at dt = 0
        float* A = reinterpret_cast<float*>(&pts[(n >> 1) * 2]);
        A[1] = 0.0f; A[3] = 0.0f; A[6] = 0.0f; A[7] = 0.0f;
        dt64[n] = 0.0;
    }
    swx2 = block_sum(swx2, red);
    if (fixs) wtot = block_sum(wtot, red);
    if (threadIdx.x == 0) {
        // per-curve terms of the incremental fold's window (see make_fold_const_inc),
        // coefficients of E rounded up to FP32
        const double dtm = __dsub_rn(tmax, tmin), df = cd->df;
        const bool uni = cd->freqs == nullptr && df > 0.0 && isfinite(df);
        const double dFd = uni ? df * pow2(96 - fxs) : 0.0;
        cd->incok = uni && dFd < 9223372036854775808.0;
        cd->dF = cd->incok ? __double2ull_rn(dFd) : 0ull;
        cd->ewc = __double2float_ru(pow2(-(fxs + 1)));
        cd->ew0 = __double2float_ru(dtm * pow2(fxs - 65) + pow2(-66) + pow2(-52));
        cd->ewt = __double2float_ru(pow2(-33) + (uni ? df : 0.0) * pow2(-(fxs + 1)) +
                                    dtm * pow2(fxs - 97) + pow2(-98));
        cd->ewh = __double2float_ru(dtm * pow2(-51) * 1.0101);
        cd->ewf = __double2float_ru(dtm * pow2(-52));
        cd->wq = fixs && wtot > 0.0 ? __double2float_rn(__ddiv_rn(1.0, wtot)) : 0.0f;
        cd->xq = fixs ? __double2float_rn(__ddiv_rn(1.0, Sx)) : 0.0f;
        cd->t_ref = tmin;
        cd->W = W;
        cd->ybar = ybar;
        cd->sumwx2 = swx2;
        cd->dtmax = __dsub_rn(tmax, tmin);
        cd->fxs = fxs;
    }
}

cudaError_t launch_prep(CurveDesc* d_curves, const int* slots, int ncurves, int* err, int phase,
                        int sums, cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    prep_kernel<<<ncurves, kPrepThreads, 0, s>>>(d_curves, slots, err, phase, sums);
    return cudaGetLastError();
}

// FP64 copies of w and w*x for the plain baseline.
__global__ void __launch_bounds__(kPrepThreads) prep_f64_kernel(const CurveDesc* curves,
                                                                 double* w64, double* wx64)
{
    const CurveDesc cd = curves[blockIdx.x];
    for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
        double inv = 1.0;
        if (cd.dy) { double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
        double w = __ddiv_rn(inv, cd.W);
        w64[cd.pt_off + i] = w;
        wx64[cd.pt_off + i] = __dmul_rn(w, __dsub_rn((double)cd.y[i], cd.ybar));
    }
}

cudaError_t launch_prep_f64(const CurveDesc* d_curves, int ncurves, double* w64, double* wx64,
                            cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    prep_f64_kernel<<<ncurves, kPrepThreads, 0, s>>>(d_curves, w64, wx64);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- a4: binning

// Histogram entry of one thread: (sum w, sum w x) as an FP32 pair, 8 bytes; the Kahan
// variant adds the two compensation terms, 16 bytes; the fixed-point variant holds the
// integer sums (sum W, sum X) as two 32-bit words, 8 bytes.  Thread t's bin b lives at entry
// b * stride + t, so the 32 lanes of a warp touch 32 consecutive entries whatever their
// bins are (no bank conflicts).

__device__ __forceinline__ void kahan_add(float4* hp, float w, float wx)
{
    float4 v = *hp;
    const float yw = __fsub_rn(w, v.z), tw = __fadd_rn(v.x, yw);
    v.z = __fsub_rn(__fsub_rn(tw, v.x), yw);
    v.x = tw;
    const float yx = __fsub_rn(wx, v.w), tx = __fadd_rn(v.y, yx);
    v.w = __fsub_rn(__fsub_rn(tx, v.y), yx);
    v.y = tx;
    *hp = v;
}

__device__ __forceinline__ u64 lds64(unsigned addr)
{
    u64 v;
    asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr));
    return v;
}
__device__ __forceinline__ void sts64(unsigned addr, u64 v)
{
    asm volatile("st.shared.b64 [%0], %1;" ::"r"(addr), "l"(v));
}
// A Kahan histogram entry (sum w, sum w x, comp w, comp w x) as two packed pairs.
__device__ __forceinline__ void lds128(unsigned addr, u64& h, u64& c)
{
    asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(h), "=l"(c) : "r"(addr));
}
__device__ __forceinline__ void sts128(unsigned addr, u64 h, u64 c)
{
    asm volatile("st.shared.v2.b64 [%0], {%1, %2};" ::"r"(addr), "l"(h), "l"(c));
}
// Kahan-compensated addition of q to the pair sums h with compensations c (both components
// at once, as kahan_add does for one): y = q - c, t = h + y, c = (t - h) - y, h = t.
__device__ __forceinline__ void kahan2(u64& h, u64& c, u64 q)
{
    const u64 y = sub2(q, c);
    const u64 t = add2(h, y);
    c = sub2(sub2(t, h), y);
    h = t;
}

// Bins of the 8 point pairs of a 16-point sub-chunk, with their weight pairs; returns
// whether any bin is not certain (then fix_sub must run before the bins are used).
template <int PHASE, bool INC, bool POW2 = false>
__device__ __forceinline__ bool fold_sub(const float4* cp, const FoldConst& fc, const FoldPacked& fq,
                                         unsigned* b, float4* Bw)
{
    bool edge = false;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 A = cp[2 * q];
        Bw[q] = cp[2 * q + 1];
        bool e0, e1;
        if (PHASE == kPhaseFX64) fold_fx_pair<INC, POW2>(A, fc, b[2 * q], b[2 * q + 1], e0, e1);
        else fold_df32_pair(A, fq, b[2 * q], b[2 * q + 1], e0, e1);
        edge = edge | e0 | e1;
    }
    return edge;
}

// Rare path: re-fold in FP64 the points of a sub-chunk whose bin is not certain.
template <int PHASE, bool INC, bool POW2 = false>
__device__ __forceinline__ void fix_sub(const float4* cp, const double* cd, const FoldConst& fc,
                                     const FoldPacked& fq, unsigned* b)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        unsigned b0, b1;
        bool e0, e1;
        if (PHASE == kPhaseFX64) fold_fx_pair<INC, POW2>(cp[2 * q], fc, b0, b1, e0, e1);
        else fold_df32_pair(cp[2 * q], fq, b0, b1, e0, e1);
        if (e0) b[2 * q] = fold_exact(cd[2 * q], fc.f, fc.nb);
        if (e1) b[2 * q + 1] = fold_exact(cd[2 * q + 1], fc.f, fc.nb);
    }
}

// Shared-memory integer reduction (no value returned).  Integer additions are exact and
// commutative, so the sums of a bin do not depend on the order of its points.
__device__ __forceinline__ void red_u32(unsigned addr, unsigned v)
{
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

// Fixed-point sums: each of the 16 points of a sub-chunk adds its (W, X) words to its bin
// with two shared-memory reductions.  A point's addition does not wait for the bin's
// previous value, and points that share a bin need no merging.
__device__ __forceinline__ void red_sub(unsigned hbase, unsigned rowb, const unsigned* b,
                                        const float4* Bw, unsigned nbu, int* err)
{
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const unsigned a = hbase + (bls_ok(b[i] < nbu, err) ? b[i] : 0u) * rowb;
        const float4& w = Bw[i >> 1];
        red_u32(a, __float_as_uint((i & 1) ? w.z : w.x));
        red_u32(a + 4u, __float_as_uint((i & 1) ? w.w : w.y));
    }
}

// The FP32 pair (r, s) of a fixed-point bin entry (W, X): r = W wq, s = X xq.
__device__ __forceinline__ void fixed_pair(u64 h, float wq, float xq, float& r, float& s)
{
    r = __fmul_rn(__uint2float_rn((unsigned)h), wq);
    s = __fmul_rn(__int2float_rn((int)(unsigned)(h >> 32)), xq);
}

// Rewrites one histogram column of nb fixed-point entries as FP32 pairs, in place.
__device__ __forceinline__ void fixed_to_f32(unsigned hbase, unsigned rowb, int nb, float wq,
                                             float xq)
{
    for (int b = 0; b < nb; ++b) {
        const unsigned a = hbase + (unsigned)b * rowb;
        float r, sx;
        fixed_pair(lds64(a), wq, xq, r, sx);
        sts64(a, pk(r, sx));
    }
}

// Read-modify-write of the 16 points of a sub-chunk in groups of kRmwGroup: all bins of a
// group are read before any is written.  Points of a group that share a bin are merged
// before the read: each point's addend is its own weights plus those of the earlier points
// of the group in its bin, so the last of them stores the bin's full total (the earlier
// stores are overwritten).  The addends depend only on the fold, so the loaded value feeds
// one packed add and the store; a bin hit by several points of one group receives their
// pre-summed weights in one addition.
constexpr int kRmwGroup = 4;

__device__ __forceinline__ void rmw_sub(unsigned hbase, unsigned rowb, const unsigned* b,
                                        const float4* Bw, unsigned nbu, int* err)
{
    constexpr int G = kRmwGroup;
#pragma unroll
    for (int g = 0; g < 16 / G; ++g) {
        const unsigned* bg = b + G * g;
        unsigned a[G];
        u64 h[G], q[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            a[i] = hbase + (bls_ok(bg[i] < nbu, err) ? bg[i] : 0u) * rowb;
            h[i] = lds64(a[i]);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const float4& w = Bw[(G * g + i) >> 1];
            q[i] = (i & 1) ? pk(w.z, w.w) : pk(w.x, w.y);
        }
        // later points first, so that every q[j] added is still a single point's weights
#pragma unroll
        for (int i = G - 1; i > 0; --i) {
#pragma unroll
            for (int j = 0; j < i; ++j) q[i] = add2_if_eq(q[i], q[j], bg[i], bg[j]);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) sts64(a[i], add2(h[i], q[i]));
    }
}

// As rmw_sub for a Kahan histogram (16-byte entries): the merged addend of each point is
// added with compensation.
__device__ __forceinline__ void rmw_sub_k(unsigned hbase, unsigned rowb, const unsigned* b,
                                          const float4* Bw, unsigned nbu, int* err)
{
    constexpr int G = kRmwGroup;
#pragma unroll
    for (int g = 0; g < 16 / G; ++g) {
        const unsigned* bg = b + G * g;
        unsigned a[G];
        u64 h[G], c[G], q[G];
#pragma unroll
        for (int i = 0; i < G; ++i) {
            a[i] = hbase + (bls_ok(bg[i] < nbu, err) ? bg[i] : 0u) * rowb;
            lds128(a[i], h[i], c[i]);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const float4& w = Bw[(G * g + i) >> 1];
            q[i] = (i & 1) ? pk(w.z, w.w) : pk(w.x, w.y);
        }
#pragma unroll
        for (int i = G - 1; i > 0; --i) {
#pragma unroll
            for (int j = 0; j < i; ++j) q[i] = add2_if_eq(q[i], q[j], bg[i], bg[j]);
        }
#pragma unroll
        for (int i = 0; i < G; ++i) {
            kahan2(h[i], c[i], q[i]);
            sts128(a[i], h[i], c[i]);
        }
    }
}

// Bins nsub staged 16-point sub-chunks into this thread's histogram (FP32 sums, point
// order).  Software pipeline: the next sub-chunk's points are loaded and folded (8
// independent pairs) in the same basic block as the current sub-chunk's read-modify-write
// chain, so the fold arithmetic fills the shared-memory latency of the chain; the rare
// FP64 re-fold runs after the stores.  hbase is the shared-memory address of this
// thread's bin 0, rowb the byte stride between bins.
template <int SUMS>
__device__ __forceinline__ void hist_sub(unsigned hbase, unsigned rowb, const unsigned* b,
                                         const float4* Bw, unsigned nbu, int* err)
{
    if (SUMS == kSumKahan) rmw_sub_k(hbase, rowb, b, Bw, nbu, err);
    else if (SUMS == kSumFixed) red_sub(hbase, rowb, b, Bw, nbu, err);
    else rmw_sub(hbase, rowb, b, Bw, nbu, err);
}

template <int PHASE, bool PINGPONG, bool INC, int SUMS = kSumF32, bool POW2 = false>
__device__ __forceinline__ void bin_fast(const float4* cp, const double* cd, int nsub,
                                         unsigned hbase, unsigned rowb, const FoldConst& fc,
                                         const FoldPacked& fq, int* err)
{
    const unsigned nbu = (unsigned)fc.nb;
    unsigned b0[16], b1[16];
    float4 W0[8], W1[8];
    if (fold_sub<PHASE, INC, POW2>(cp, fc, fq, b0, W0)) fix_sub<PHASE, INC, POW2>(cp, cd, fc, fq, b0);
    int sc = 0;
    if (PINGPONG) {
        // the two buffers used in turn (the loop body covers two sub-chunks): no register
        // copies between sub-chunks (faster in the warp-specialised kernel, whose binning
        // warps are the critical path; slower in the one-group kernel)
        for (; sc + 2 < nsub; sc += 2) {
            const float4* n1 = cp + 16 * (sc + 1);
            const bool e1 = fold_sub<PHASE, INC, POW2>(n1, fc, fq, b1, W1);
            hist_sub<SUMS>(hbase, rowb, b0, W0, nbu, err);
            if (e1) fix_sub<PHASE, INC, POW2>(n1, cd + 16 * (sc + 1), fc, fq, b1);
            const float4* n2 = cp + 16 * (sc + 2);
            const bool e2 = fold_sub<PHASE, INC, POW2>(n2, fc, fq, b0, W0);
            hist_sub<SUMS>(hbase, rowb, b1, W1, nbu, err);
            if (e2) fix_sub<PHASE, INC, POW2>(n2, cd + 16 * (sc + 2), fc, fq, b0);
        }
    }
    for (; sc + 1 < nsub; ++sc) {
        const float4* n1 = cp + 16 * (sc + 1);
        const bool e1 = fold_sub<PHASE, INC, POW2>(n1, fc, fq, b1, W1);
        hist_sub<SUMS>(hbase, rowb, b0, W0, nbu, err);
        if (e1) fix_sub<PHASE, INC, POW2>(n1, cd + 16 * (sc + 1), fc, fq, b1);
#pragma unroll
        for (int i = 0; i < 16; ++i) b0[i] = b1[i];
#pragma unroll
        for (int q = 0; q < 8; ++q) W0[q] = W1[q];
    }
    hist_sub<SUMS>(hbase, rowb, b0, W0, nbu, err);
}

// Generic binning (FP64 or FP32 phase modes, precision studies): pair by pair.
template <int PHASE, int SUMS = kSumF32>
__device__ __forceinline__ void bin_generic(const float4* cp, const double* cd, int npairs,
                                            unsigned hbase, unsigned rowb, const FoldConst& fc,
                                            const FoldPacked& fq, int* err)
{
    for (int pi = 0; pi < npairs; ++pi) {
        const float4 A = cp[2 * pi], B = cp[2 * pi + 1];
        unsigned b0, b1;
        fold_pair<PHASE>(A, &cd[2 * pi], fc, fq, b0, b1);
        const unsigned nbu = (unsigned)fc.nb;
        const unsigned a0 = hbase + (bls_ok(b0 < nbu, err) ? b0 : 0u) * rowb;
        const unsigned a1 = hbase + (bls_ok(b1 < nbu, err) ? b1 : 0u) * rowb;
        if (SUMS == kSumFixed) {
            red_u32(a0, __float_as_uint(B.x));
            red_u32(a0 + 4u, __float_as_uint(B.y));
            red_u32(a1, __float_as_uint(B.z));
            red_u32(a1 + 4u, __float_as_uint(B.w));
        } else if (SUMS == kSumKahan) {
            u64 h, c;
            lds128(a0, h, c);
            kahan2(h, c, pk(B.x, B.y));
            sts128(a0, h, c);
            lds128(a1, h, c);
            kahan2(h, c, pk(B.z, B.w));
            sts128(a1, h, c);
        } else {
            sts64(a0, add2(lds64(a0), pk(B.x, B.y)));
            sts64(a1, add2(lds64(a1), pk(B.z, B.w)));
        }
    }
}

// ------------------------------------------------------------------------- a5/a6: sweep

__device__ __forceinline__ float bin_w(const unsigned char* hist, size_t S, int kahan, int b)
{
    if (kahan) {
        const float4 v = reinterpret_cast<const float4*>(hist)[(size_t)b * S];
        return __fsub_rn(v.x, v.z);
    }
    return reinterpret_cast<const float2*>(hist)[(size_t)b * S].x;
}

__device__ __forceinline__ float bin_x(const unsigned char* hist, size_t S, int kahan, int b)
{
    if (kahan) {
        const float4 v = reinterpret_cast<const float4*>(hist)[(size_t)b * S];
        return __fsub_rn(v.y, v.w);
    }
    return reinterpret_cast<const float2*>(hist)[(size_t)b * S].y;
}

// Fast sweep: the largest power P of any box, without its position.
//
// SB consecutive starts share every bin load; their sums are carried as SB/2 packed pairs
// (one f32x2 instruction updates two starts).  Conditions: kmax - kmin + 1 >= SB - 1, and
// no box can hold more than 0.89 of the weight (checked by the caller).  The starts of the
// last block may pass nb; they repeat earlier starts and cannot change the maximum.
//
// Fast-sweep evaluation of two boxes (starts 2q and 2q+1 of a block) that grow by one bin.
// R holds -r of the two boxes and X their s; d = r(1-r) comes from one fused rounding,
// -d = r^2 - r.  The fast sweep only runs where every box has r < 0.89, so d > 0.  Two
// forms rank the boxes, with different shares of special-function and FP32 work:
//
// FORM 0, signed residue: z = s * rsqrt(d) (P = z^2), one approximate reciprocal square
// root per box and one product.  Dips (SIGN = 0) are the boxes with s < 0, so the most
// negative z wins; with both signs the largest |z| does.  An empty box (r = 0, s = 0
// exactly) gives 0 * inf = NaN, which min/max ignore.
//
// FORM 1, power with a shared reciprocal: 1/(d0 d1) gives 1/d0 = d1/(d0 d1) and
// 1/d1 = d0/(d0 d1), one reciprocal for the two boxes; P = s^2/d (dips: -s|s|/d, negative
// for bumps).  An empty box would make the shared product zero, so its -r starts at
// -kEmptyBox instead of 0: d0 d1 >= kEmptyBox^2 stays a normal FP32 number, an empty box
// evaluates to P = 0, and for a real box (r >= 1e-10, far below one point's weight in
// practice) the offset is below half an ulp of r and changes nothing.
//
// Both approximations err by about 2^-22 relative, far inside the spectrum's tolerance.
constexpr float kEmptyBox = 1e-18f;

// Three-input FP32 min / max (NaN inputs are ignored, as by fminf / fmaxf).
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

template <int SIGN, int FORM, bool SEED>
__device__ __forceinline__ void eval_pair(u64& R, u64& X, const u64& HW2, const u64& HX2,
                                          bool init, bool use0, bool use1, float& b0, float& b1)
{
    if (init) {
        // the second start of the pair begins at the next bin; with SEED, (R, X) already
        // hold the starts' seeds (see sweep_fast)
        float hw, hw1, hx, hx1;
        upk(HW2, hw, hw1);
        upk(HX2, hx, hx1);
        if (SEED) {
            R = sub2(R, pk(hw, 0.0f));
            X = add2(X, pk(hx, 0.0f));
        } else {
            R = FORM ? pk(-hw - kEmptyBox, -kEmptyBox) : pk(-hw, 0.0f);
            X = pk(hx, 0.0f);
        }
    } else {
        R = sub2(R, HW2);
        X = add2(X, HX2);
    }
    const u64 ND = fma2(R, R, R);   // (r0^2 - r0, r1^2 - r1) = (-d0, -d1)
    float nd0, nd1;
    upk(ND, nd0, nd1);
    if (FORM == 0) {
        const u64 Z = mul2(X, pk(rsqrt_approx(-nd0), rsqrt_approx(-nd1)));
        float z0, z1;
        upk(Z, z0, z1);
        if (use0 && use1) {   // both boxes count: one three-input min/max for the pair
            b0 = SIGN ? fmax3(b0, fabsf(z0), fabsf(z1)) : fmin3(b0, z0, z1);
        } else if (SIGN) {
            if (use0) b0 = fmaxf(b0, fabsf(z0));
            if (use1) b1 = fmaxf(b1, fabsf(z1));
        } else {
            if (use0) b0 = fminf(b0, z0);
            if (use1) b1 = fminf(b1, z1);
        }
    } else {
        const float rc = rcp_approx(nd0 * nd1);
        const u64 Q = mul2(X, pk(nd1 * rc, nd0 * rc));   // (-s0/d0, -s1/d1)
        float q0, q1, s0, s1;
        upk(Q, q0, q1);
        upk(X, s0, s1);
        const float p0 = SIGN ? q0 * -s0 : q0 * fabsf(s0);
        const float p1 = SIGN ? q1 * -s1 : q1 * fabsf(s1);
        if (use0) b0 = fmaxf(b0, p0);
        if (use1) b1 = fmaxf(b1, p1);
    }
}

// One step of the fast sweep over one block: bin value (hw, hx) for the pairs [Q0, Q1),
// with the ramp rules given by (init, use0, use1) per pair (see sweep_fast).
template <int SIGN, int NP, int FORM, bool SEED>
__device__ __forceinline__ void sweep_step(float hw, float hx, u64* R, u64* X, float* b0,
                                           float* b1, int mm, int phase, int e)
{
    const u64 HW2 = pk(hw, hw), HX2 = pk(hx, hx);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        if (phase == 0) {          // ramp-up at bin mm
            if (2 * q > mm) continue;
            eval_pair<SIGN, FORM, SEED>(R[q], X[q], HW2, HX2, 2 * q == mm, true, 2 * q < mm, b0[q], b1[q]);
        } else if (phase == 1) {   // steady
            eval_pair<SIGN, FORM, SEED>(R[q], X[q], HW2, HX2, false, true, true, b0[q], b1[q]);
        } else {                   // ramp-down step e
            if (2 * q + 1 < e + 1) continue;
            eval_pair<SIGN, FORM, SEED>(R[q], X[q], HW2, HX2, false, 2 * q >= e + 1, true, b0[q], b1[q]);
        }
    }
}

#ifndef BLS_SWEEP_MIX
#define BLS_SWEEP_MIX 1
#endif
// Form of block B (block A always uses the signed residue): mixing the two balances the
// special-function unit against the FP32 pipe.
constexpr int kFormB = BLS_SWEEP_MIX;

// Bin sources of the fast sweep.  start(a, b) places block A at bin a and block B at bin
// b; next() returns the next bin of each block; finish() ends a block.
//
// SmemBins reads the private histogram column in shared memory, cyclically.
struct SmemBins {
    unsigned hbase, rowb;
    int nb, ma, mb;
    int* err = nullptr;
    __device__ __forceinline__ void start(int a, int b) { ma = a; mb = b; }
    __device__ __forceinline__ void next(float& hwa, float& hxa, float& hwb, float& hxb)
    {
        if (!bls_ok((unsigned)ma < (unsigned)nb && (unsigned)mb < (unsigned)nb, err)) ma = mb = 0;
        upk(lds64(hbase + (unsigned)ma * rowb), hwa, hxa);
        upk(lds64(hbase + (unsigned)mb * rowb), hwb, hxb);
        ma = (ma + 1 == nb) ? 0 : ma + 1;
        mb = (mb + 1 == nb) ? 0 : mb + 1;
    }
    __device__ __forceinline__ void finish() {}
};

// Tensor-memory access of this thread's own lane (shape 32x32b: lane i of the warp reads
// or writes TMEM lane base + i, the address's column field selects 32-bit columns).  The
// loads complete asynchronously; tmem_wait_ld4 takes the destination registers as
// operands, so no use of them can be scheduled before the wait.
__device__ __forceinline__ void tmem_ld2(unsigned ta, unsigned& v0, unsigned& v1)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];"
                 : "=r"(v0), "=r"(v1) : "r"(ta));
}
__device__ __forceinline__ void tmem_wait_ld4(unsigned& a, unsigned& b, unsigned& c, unsigned& d)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(a), "+r"(b), "+r"(c), "+r"(d));
}
__device__ __forceinline__ void tmem_st16(unsigned ta, const unsigned* v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, "
                 "%9, %10, %11, %12, %13, %14, %15, %16};"
                 :: "r"(ta), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
                    "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]),
                    "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// TmemBins reads a copy of the histogram column in this thread's TMEM lane: bin b at
// columns (2b, 2b + 1), laid out linearly past nb (bins nb.. repeat bins 0..), so a block
// reads consecutive columns; with WRAP the copy holds bins 0 .. nb-1 only and the reads
// wrap at nb (for nb too large for the repeated bins).  The next bin of both blocks is
// always in flight while the current one is evaluated.
template <bool WRAP>
struct TmemBins {
    unsigned base, tend, ta, tb;   // tend: column 2 nb (WRAP: the copy holds bins 0..nb-1 only)
    unsigned pa0, pa1, pb0, pb1;
    int* err = nullptr;
    __device__ __forceinline__ void issue()
    {
        // the two columns read at ta and at tb lie in the 512-column allocation
        if (!bls_ok(ta - base <= 510u && tb - base <= 510u, err)) ta = tb = base;
        tmem_ld2(ta, pa0, pa1);
        tmem_ld2(tb, pb0, pb1);
        ta += 2;
        tb += 2;
        if (WRAP) {
            ta = ta == tend ? base : ta;
            tb = tb == tend ? base : tb;
        }
    }
    __device__ __forceinline__ void start(int a, int b)
    {
        ta = base + 2u * (unsigned)a;
        tb = base + 2u * (unsigned)b;
        issue();
    }
    __device__ __forceinline__ void next(float& hwa, float& hxa, float& hwb, float& hxb)
    {
        tmem_wait_ld4(pa0, pa1, pb0, pb1);
        hwa = __uint_as_float(pa0);
        hxa = __uint_as_float(pa1);
        hwb = __uint_as_float(pb0);
        hxb = __uint_as_float(pb1);
        issue();
    }
    __device__ __forceinline__ void finish() { tmem_wait_ld4(pa0, pa1, pb0, pb1); }
};

// Fast sweep over two independent blocks of SB starts at a time (starts i0.. and
// i0 + half..), so that 2*SB/2 packed pairs are in flight per bin step.  Block A covers
// starts [0, half), block B [half, 2 half) with half = SB * ceil(nb / (2 SB)); starts past
// nb repeat earlier ones (cyclic) and cannot change the maximum.  The outer steps i0 are
// dealt round-robin to `nparts` threads sharing the histogram; `part` is this thread's.
// Widths kmin .. kmax: every box of start s holds bins s .. s + kmin - 2, whose sums (in
// bin order) seed the start's running sums, and the steps then run over the kx = kmax -
// kmin + 1 widths as for kmin = 1.  A block reads SB + kmin - 2 bins for the seeds (when
// kmin > 1) and kx + SB - 1 bins from its start + kmin - 1 (cyclic).  FB is the form of
// block B.  Condition: kx >= SB - 1.
template <int SB, int SIGN, class Bins, int FB, bool SEED>
__device__ __forceinline__ float sweep_fast_t(Bins& src, int nb, int kmin, int kmax, int part,
                                              int nparts)
{
    constexpr int NP = SB / 2;
    const int kx = kmax - kmin + 1;
    float a0[NP], a1[NP], c0[NP], c1[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q) { a0[q] = 0.0f; a1[q] = 0.0f; c0[q] = 0.0f; c1[q] = 0.0f; }
    const int half = SB * ((nb + 2 * SB - 1) / (2 * SB));
    for (int i0 = part * SB; i0 < half; i0 += nparts * SB) {
        // R holds -r (the form-1 block offset by -kEmptyBox, see eval_pair), X holds s;
        // with kmin > 1 both start from the seeds: start s (s = 0 .. SB-1 of the block)
        // takes bins s .. s + kmin - 2, in bin order
        const u64 r0B = FB ? pk(-kEmptyBox, -kEmptyBox) : 0ull;
        u64 RA[NP], XA[NP], RB[NP], XB[NP];
#pragma unroll
        for (int q = 0; q < NP; ++q) { RA[q] = 0ull; XA[q] = 0ull; RB[q] = r0B; XB[q] = 0ull; }
        int mb = i0 + half;
        while (mb >= nb) mb -= nb;
        if (SEED) {
            src.start(i0, mb);
            for (int m = 0; m < SB + kmin - 2; ++m) {
                float hwa, hxa, hwb, hxb;
                src.next(hwa, hxa, hwb, hxb);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const bool t0 = m >= 2 * q && m <= 2 * q + kmin - 2;
                    const bool t1 = m >= 2 * q + 1 && m <= 2 * q + kmin - 1;
                    RA[q] = sub2(RA[q], pk(t0 ? hwa : 0.0f, t1 ? hwa : 0.0f));
                    XA[q] = add2(XA[q], pk(t0 ? hxa : 0.0f, t1 ? hxa : 0.0f));
                    RB[q] = sub2(RB[q], pk(t0 ? hwb : 0.0f, t1 ? hwb : 0.0f));
                    XB[q] = add2(XB[q], pk(t0 ? hxb : 0.0f, t1 ? hxb : 0.0f));
                }
            }
            src.finish();
        }
        int ma = i0 + kmin - 1, mc = mb + kmin - 1;
        while (ma >= nb) ma -= nb;
        while (mc >= nb) mc -= nb;
        src.start(ma, mc);
#pragma unroll
        for (int mm = 0; mm < SB - 1; ++mm) {
            float hwa, hxa, hwb, hxb;
            src.next(hwa, hxa, hwb, hxb);
            sweep_step<SIGN, NP, 0, SEED>(hwa, hxa, RA, XA, a0, a1, mm, 0, 0);
            sweep_step<SIGN, NP, FB, SEED>(hwb, hxb, RB, XB, c0, c1, mm, 0, 0);
        }
#pragma unroll 2
        for (int mm = SB - 1; mm < kx; ++mm) {
            float hwa, hxa, hwb, hxb;
            src.next(hwa, hxa, hwb, hxb);
            sweep_step<SIGN, NP, 0, SEED>(hwa, hxa, RA, XA, a0, a1, 0, 1, 0);
            sweep_step<SIGN, NP, FB, SEED>(hwb, hxb, RB, XB, c0, c1, 0, 1, 0);
        }
#pragma unroll
        for (int e = 0; e < SB - 1; ++e) {
            float hwa, hxa, hwb, hxb;
            src.next(hwa, hxa, hwb, hxb);
            sweep_step<SIGN, NP, 0, SEED>(hwa, hxa, RA, XA, a0, a1, 0, 2, e);
            sweep_step<SIGN, NP, FB, SEED>(hwb, hxb, RB, XB, c0, c1, 0, 2, e);
        }
        src.finish();
    }
    // best signed residue of block A -> power P = z^2; block B holds powers or residues
    float za = 0.0f, zb = 0.0f, pb = 0.0f;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
        za = SIGN ? fmaxf(za, fmaxf(a0[q], a1[q])) : fminf(za, fminf(a0[q], a1[q]));
        if (FB) pb = fmaxf(pb, fmaxf(c0[q], c1[q]));
        else zb = SIGN ? fmaxf(zb, fmaxf(c0[q], c1[q])) : fminf(zb, fminf(c0[q], c1[q]));
    }
    return fmaxf(fmaxf(za * za, zb * zb), pb);
}

// The fast sweep; kmin > 1 takes the seeded variant (a separate instantiation, so that the
// common kmin = 1 case keeps its registers).
template <int SB, int SIGN, class Bins, int FB = kFormB>
__device__ __forceinline__ float sweep_fast(Bins& src, int nb, int kmin, int kmax, int part,
                                            int nparts)
{
    return kmin > 1 ? sweep_fast_t<SB, SIGN, Bins, FB, true>(src, nb, kmin, kmax, part, nparts)
                    : sweep_fast_t<SB, SIGN, Bins, FB, false>(src, nb, kmin, kmax, part, nparts);
}

struct Best {
    float num, den;   // P = num / den
    int i1, k;
};

__device__ __forceinline__ bool box_full(int i1, int k, int nb, int arc_a, int arc_len)
{
    int rel = arc_a - i1;
    if (rel < 0) rel += nb;
    return rel + arc_len <= k;
}

// Sequential bin stream over a shared-memory histogram column (cyclic).
struct SmemStream {
    const unsigned char* hist;
    size_t S;
    int kahan, nb, m;
    __device__ __forceinline__ void start(int a) { m = a; }
    __device__ __forceinline__ void next(float& hw, float& hx)
    {
        hw = bin_w(hist, S, kahan, m);
        hx = bin_x(hist, S, kahan, m);
        m = (m + 1 == nb) ? 0 : m + 1;
    }
    __device__ __forceinline__ void finish() {}
};

// Exact sweep: the best box with the definition's tie-break.
//
// Every start i1 and width k (cyclic), sums accumulated bin by bin from the start: r in
// double-FP32 (so 1 - r stays accurate when the box holds most of the weight), s with
// Kahan compensation.  A box counts when it holds at least one point and leaves one out:
// an empty box has r = 0 exactly, and a box holding every point contains the shortest
// cyclic arc of occupied bins, so neither depends on rounding.  Dips only: s < 0.
// Candidates are compared as exact (num, den) pairs, num * den_best > num_best * den, so a
// box with bit-identical sums never replaces an earlier one and equal powers resolve to
// the smallest (i1, k).  The bins come from a sequential stream (start, next, finish).
// With PART, only the starts i1 = i1_first, i1_first + i1_step, ... are swept (a share of
// the starts for one of several threads; their results meet in better_box).
template <int SIGN, class Stream, bool PART = false>
__device__ Best sweep_exact_src(Stream& src, int nb, int kmin, int kmax, int i1_first = 0,
                                int i1_step = 1)
{
    int first = -1, last = -1, run = 0, gap = 0, gap_end = 0;
    src.start(0);
    for (int b = 0; b < nb; ++b) {
        float hw, hx;
        src.next(hw, hx);
        if (hw != 0.0f) {
            if (first < 0) first = b;
            else if (run > gap) { gap = run; gap_end = b; }
            last = b;
            run = 0;
        } else if (first >= 0) {
            ++run;
        }
    }
    src.finish();
    int arc_a = 0, arc_len = 0;
    if (first >= 0) {
        const int wrap = (nb - 1 - last) + first;
        if (wrap >= gap) { arc_a = first; arc_len = last - first + 1; }
        else { arc_a = gap_end; arc_len = nb - gap; }
    }
    Best g;
    g.num = 0.0f; g.den = 1.0f; g.i1 = 0; g.k = kmin;
    for (int i1 = PART ? i1_first : 0; i1 < nb; i1 += PART ? i1_step : 1) {
        float rh = 0.0f, rl = 0.0f, s = 0.0f, cs = 0.0f;
        src.start(i1);
        for (int k = 1; k <= kmax; ++k) {
            float hw, hx;
            src.next(hw, hx);
            const float t = __fadd_rn(rh, hw);                      // two-sum rh + hw
            const float bp = __fsub_rn(t, rh);
            const float e = __fadd_rn(__fsub_rn(rh, __fsub_rn(t, bp)), __fsub_rn(hw, bp));
            rh = t;
            rl = __fadd_rn(rl, e);
            const float y = __fsub_rn(hx, cs), ts = __fadd_rn(s, y);  // Kahan s + hx
            cs = __fsub_rn(__fsub_rn(ts, s), y);
            s = ts;
            if (k < kmin || rh == 0.0f) continue;
            if (box_full(i1, k, nb, arc_a, arc_len)) continue;
            const float q = __fsub_rn(__fsub_rn(1.0f, rh), rl);     // 1 - r
            const float den = __fmaf_rn(rh, q, __fmul_rn(rl, q));    // r (1 - r)
            if (!(den > 0.0f)) continue;
            const float num = SIGN ? __fmul_rn(s, s) : __fmul_rn(-s, fabsf(s));
            if (__fmul_rn(num, g.den) > __fmul_rn(g.num, den)) {
                g.num = num; g.den = den; g.i1 = i1; g.k = k;
            }
        }
        src.finish();
    }
    return g;
}

template <int SIGN>
__device__ Best sweep_exact(const unsigned char* hist, int stride, int kahan, int nb, int kmin,
                            int kmax)
{
    SmemStream src;
    src.hist = hist;
    src.S = (size_t)stride;
    src.kahan = kahan;
    src.nb = nb;
    return sweep_exact_src<SIGN>(src, nb, kmin, kmax);
}

__device__ __forceinline__ Best sweep_exact_rt(int sign, const unsigned char* hist, int stride,
                                               int kahan, int nb, int kmin, int kmax)
{
    return sign ? sweep_exact<1>(hist, stride, kahan, nb, kmin, kmax)
                : sweep_exact<0>(hist, stride, kahan, nb, kmin, kmax);
}

// Whether candidate h beats g under the exact sweep's order: the larger power (compared as
// num_h den_g > num_g den_h, as the sweep compares), equal cross products to the smaller
// (i1, k).
__device__ __forceinline__ bool better_box(const Best& h, const Best& g)
{
    const float a = __fmul_rn(h.num, g.den), b = __fmul_rn(g.num, h.den);
    return a > b || (a == b && (h.i1 < g.i1 || (h.i1 == g.i1 && h.k < g.k)));
}

// The exact sweep by the 32 lanes of a warp: lane l sweeps the starts l, l + 32, ..., then
// the lanes' bests meet by shuffles under better_box.  Every lane returns the result.
template <int SIGN>
__device__ Best sweep_exact_warp(const unsigned char* hist, int stride, int kahan, int nb,
                                 int kmin, int kmax, int lane)
{
    SmemStream src;
    src.hist = hist;
    src.S = (size_t)stride;
    src.kahan = kahan;
    src.nb = nb;
    Best g = sweep_exact_src<SIGN, SmemStream, true>(src, nb, kmin, kmax, lane, 32);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Best h;
        h.num = __shfl_xor_sync(0xffffffffu, g.num, o);
        h.den = __shfl_xor_sync(0xffffffffu, g.den, o);
        h.i1 = __shfl_xor_sync(0xffffffffu, g.i1, o);
        h.k = __shfl_xor_sync(0xffffffffu, g.k, o);
        if (better_box(h, g)) g = h;
    }
    return g;
}

// Largest power of one private histogram: fast sweep when its conditions hold, else the
// exact sweep.  The fast sweep needs that no box holds more than 0.9 of the weight; the
// cheap test kmax * (heaviest bin) < 0.89 settles most frequencies, and when it fails the
// heaviest run of kmax bins is measured with a sliding sum (the 0.01 margin covers FP32
// rounding of the sums).
// The largest power of one frequency's histogram, or (nparts > 1) of this thread's share
// of the box starts: the fast sweep is split over the threads, the exact sweep runs on
// part 0 alone (the others return 0, below any power a box can reach).
template <int KAHAN, int SIGN, int SB>
__device__ __forceinline__ float sweep_max(const unsigned char* hist, int stride, int nb,
                                           int kmin, int kmax, int part, int nparts,
                                           int* err = nullptr)
{
    if (!KAHAN && kmax - kmin + 1 >= SB - 1) {
        const unsigned hbase = (unsigned)__cvta_generic_to_shared(hist);
        const unsigned rowb = (unsigned)stride * 8u;
        float wmax = 0.0f;
        for (int b = 0; b < nb; ++b) {
            float hw, hx;
            upk(lds64(hbase + (unsigned)b * rowb), hw, hx);
            wmax = fmaxf(wmax, hw);
        }
        bool fast = (float)kmax * wmax < 0.89f;
        if (!fast && kmax < nb) {
            float win = 0.0f, hw, hx;
            for (int b = 0; b < kmax; ++b) {
                upk(lds64(hbase + (unsigned)b * rowb), hw, hx);
                win += hw;
            }
            float rmax = win;
            int add = kmax;
            for (int b = 0; b + 1 < nb; ++b) {   // window [b+1, b+kmax] (cyclic)
                float hin, hout;
                upk(lds64(hbase + (unsigned)add * rowb), hin, hx);
                upk(lds64(hbase + (unsigned)b * rowb), hout, hx);
                win = __fsub_rn(__fadd_rn(win, hin), hout);
                rmax = fmaxf(rmax, win);
                add = (add + 1 == nb) ? 0 : add + 1;
            }
            fast = rmax < 0.89f;
        }
        if (fast) {
            SmemBins src;
            src.hbase = hbase;
            src.rowb = rowb;
            src.nb = nb;
            src.err = err;
            return sweep_fast<SB, SIGN>(src, nb, kmin, kmax, part, nparts);
        }
    }
    if (part != 0) return 0.0f;
    const Best g = sweep_exact<SIGN>(hist, stride, KAHAN, nb, kmin, kmax);
    return g.num > 0.0f ? __fdiv_rn(g.num, g.den) : 0.0f;
}

// ------------------------------------------------------------------------- a2-a6: hot kernel

// Starts per block of the fast sweep for wide boxes (kmax >= 15): 8 or 10, whichever
// wastes fewer starts once the nb starts are dealt to nparts threads in steps of two
// blocks (nb = 200 over 2 threads: 10 gives 5 + 5 steps with none wasted, 8 gives 7 + 6).
__host__ __device__ __forceinline__ bool wide_sweep_10(int nb, int nparts)
{
    const int s8 = 16 * nparts, s10 = 20 * nparts;
    return ((nb + s10 - 1) / s10) * s10 < ((nb + s8 - 1) / s8) * s8;
}

// Starts per block of the fast sweep for widths kmin .. kmax (one sweep thread per column).
__host__ __device__ __forceinline__ int sweep_block(int nb, int kmin, int kmax)
{
    return kmax - kmin + 1 < 15 ? 4 : (wide_sweep_10(nb, 1) ? 10 : 8);
}

// How the warp-specialised kernel sweeps a tile from its TMEM copy (0: it cannot, the fast
// sweep does not cover the widths or nb > 256).  1, linear: the copy repeats the first bins
// past nb, so the sweep's reads never wrap (they reach bin nb + kmax + SB - 2 with the one
// bin of read-ahead; the copy's last group of 8 up to 7 more; all within the 512 columns,
// the copy's reads past nb wrapping once).  2, wrapped: the copy holds bins 0 .. nb-1 and
// every read wraps at nb (one compare and select per bin and block).
__host__ __device__ __forceinline__ int ws_tmem_mode(int nb, int kmin, int kmax)
{
    const int SB = sweep_block(nb, kmin, kmax);
    if (kmax - kmin + 1 < SB - 1) return 0;
    if (nb + kmax + SB + 8 <= 257 && kmax + SB + 8 <= nb) return 1;
    return nb <= 256 && nb >= 8 ? 2 : 0;
}

constexpr int kFoldMaxThreads = 256;

// Shared memory of a fold-sweep block: [staging: 2 x chunk point pairs + FP64 offsets]
// [histograms: nb_max rows x stride entries].
size_t fold_smem_bytes(int T, int stride, int nb_max, int chunk, int sums)
{
    (void)T;
    size_t stage = (size_t)2 * chunk * (sizeof(float4) + sizeof(double));
    size_t hist = (size_t)nb_max * stride * hist_entry_bytes(sums);
    return stage + hist;
}

int fold_sweep_max_threads() { return kFoldMaxThreads; }

// Threads per block for `cols` frequencies per tile: two per column when they fit (the
// second one halves the sweep's share of each thread), else one.
#ifndef BLS_SWEEP_SPLIT
#define BLS_SWEEP_SPLIT 2
#endif
int fold_block_threads(int cols)
{
    return (BLS_SWEEP_SPLIT == 2 && 2 * cols <= kFoldMaxThreads) ? 2 * cols : cols;
}

template <int PHASE, int SUMS, int SIGN>
__global__ void __launch_bounds__(kFoldMaxThreads, 1) fold_sweep_kernel(FoldParams p)
{
    constexpr int KAHAN = SUMS == kSumKahan;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    // p.cols frequencies per tile, one histogram column each; blockDim.x is cols or
    // 2 cols: threads [cols, 2 cols) help stage the points and sweep the boxes of column
    // tid - cols (the binning needs one private histogram per thread and shared memory
    // holds only cols of them; the sweep only reads them)
    const int T = p.cols;
    const int NT = blockDim.x;
    const int tid = threadIdx.x;
    const int part = tid < T ? 0 : 1;
    const int col = tid - part * T;
    const int nparts = NT / T;
    const int CH = p.chunk;
    float4* cpts = reinterpret_cast<float4*>(smem);             // [2][CH]: point pairs
    double* cdt = reinterpret_cast<double*>(cpts + 2 * CH);     // [2][CH]: FP64 offsets
    unsigned char* hist_all = reinterpret_cast<unsigned char*>(cdt + 2 * CH);
    const size_t esz = KAHAN ? sizeof(float4) : sizeof(float2);
    unsigned char* hist = hist_all + (size_t)col * esz;         // column of this thread
    const size_t S = (size_t)p.stride;

    for (;;) {
        __syncthreads();
        if (tid == 0) s_item = atomicAdd(p.counter, 1);
        __syncthreads();
        const long long it = s_item;
        if (it >= p.total) break;
        int lo = 0, hi = p.nranges;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (p.prefix[mid] <= it) lo = mid; else hi = mid;
        }
        const TileRange tr = p.ranges[lo];
        const CurveDesc& cdr = p.curves[tr.curve];
        const int n = cdr.n, nf = cdr.nf, nb = cdr.nb, kmin = cdr.kmin, kmax = cdr.kmax;
        const float4* gpts = cdr.pts;
        const double* gdt = cdr.dt64;
        const int tile = tr.tile_lo + (int)(it - p.prefix[lo]);
        const int j = tile * T + col;
        const bool active = j < nf;
        const int jt = active ? j : nf - 1;
        const double f = grid_freq(cdr, jt);
        // FX64 tiles of a uniform grid (plain sums) take the incremental fold, with the
        // tile's middle column (at most its last frequency) as the reference column
        const int jc = min(tile * T + T / 2, nf - 1);
        const double fcen = grid_freq(cdr, jc);
        const bool inc = PHASE == kPhaseFX64 && !KAHAN && cdr.freqs == nullptr &&
                         inc_tile_ok(fcen, cdr);
        FoldConst fc = make_fold_const(f, nb, cdr.dtmax, cdr.fxs, !inc,
                                       PHASE == kPhaseDF32 || PHASE == kPhaseF32);
        if (inc) make_fold_const_inc(fc, f, fcen, jt - jc, cdr, nb);
        const FoldPacked fq = make_fold_packed(fc);

        for (int b = 0; b < nb && part == 0; ++b) {
            if (KAHAN)
                reinterpret_cast<float4*>(hist)[(size_t)b * S] = make_float4(0.f, 0.f, 0.f, 0.f);
            else
                reinterpret_cast<u64*>(hist)[(size_t)b * S] = 0ull;
        }

        // a2: stage the curve through shared memory in chunks of CH points (CH a multiple
        // of 16), double-buffered with cp.async; the last chunk is padded with zero-weight
        // points at dt = 0 up to a whole 16-point sub-chunk (they add +0 to bin 0)
        const int nchunks = (n + CH - 1) / CH;
        auto stage = [&](int ci) {
            const int c0 = ci * CH;
            const int cn = (min(CH, n - c0) + 1) & ~1;          // whole pairs exist in memory
            const int cpad = (cn + 15) & ~15;
            float4* dp = cpts + (ci & 1) * CH;
            double* dd = cdt + (ci & 1) * CH;
            for (int i = tid; i < cn; i += NT) {
                cp_async16(&dp[i], &gpts[c0 + i]);
                cp_async8(&dd[i], &gdt[c0 + i]);
            }
            for (int i = cn + tid; i < cpad; i += NT) {
                dp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                dd[i] = 0.0;
            }
            cp_async_commit();
        };
        const unsigned hbase = (unsigned)__cvta_generic_to_shared(hist);
        const unsigned rowb = (unsigned)(S * esz);
        stage(0);
        for (int ci = 0; ci < nchunks; ++ci) {
            if (ci + 1 < nchunks) stage(ci + 1); else cp_async_commit();
            cp_async_wait1();
            if (inc) inc_stage(cpts + (ci & 1) * CH, (min(CH, n - ci * CH) + 1) & ~1, tid, NT, fc);
            __syncthreads();
            const int cnum = min(CH, n - ci * CH);
            const float4* cp = cpts + (ci & 1) * CH;
            const double* cd = cdt + (ci & 1) * CH;
            if (active && part == 0) {   // a3 + a4: fold and bin
                if (KAHAN) {
                    const int npairs = (cnum + 1) >> 1;
                    for (int pi = 0; pi < npairs; ++pi) {
                        const float4 A = cp[2 * pi], B = cp[2 * pi + 1];
                        unsigned b0, b1;
                        fold_pair<PHASE>(A, &cd[2 * pi], fc, fq, b0, b1);
                        if (!bls_ok(b0 < (unsigned)nb && b1 < (unsigned)nb, p.err)) continue;
                        kahan_add(reinterpret_cast<float4*>(hist) + b0 * S, B.x, B.y);
                        kahan_add(reinterpret_cast<float4*>(hist) + b1 * S, B.z, B.w);
                    }
                } else if ((PHASE == kPhaseDF32 && fc.fast) || (PHASE == kPhaseFX64 && fc.fxok)) {
                    if (inc && fc.sh != 0u)
                        bin_fast<PHASE, false, true, SUMS, true>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                    else if (inc)
                        bin_fast<PHASE, false, true, SUMS>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                    else
                        bin_fast<PHASE, false, false, SUMS>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                } else {
                    bin_generic<PHASE, SUMS>(cp, cd, (cnum + 1) >> 1, hbase, rowb, fc, fq, p.err);
                }
            }
            __syncthreads();
        }
        if (SUMS == kSumFixed) {   // integer sums -> FP32 (r, s), each binning thread its column
            if (active && part == 0) fixed_to_f32(hbase, rowb, nb, cdr.wq, cdr.xq);
            __syncthreads();
        }

        // a5 + a6: box sweep; the partial maxima of a column meet in the staging buffer,
        // idle once the last chunk is binned (2 CH x 24 B >= 1536 B since CH >= 32, more
        // than the 4 B x blockDim.x <= 1024 B needed)
        float v = 0.0f;
        if (active)
            v = kmax - kmin + 1 < 15 ? sweep_max<KAHAN, SIGN, 4>(hist, p.stride, nb, kmin, kmax, part, nparts, p.err)
                : wide_sweep_10(nb, nparts)
                    ? sweep_max<KAHAN, SIGN, 10>(hist, p.stride, nb, kmin, kmax, part, nparts, p.err)
                    : sweep_max<KAHAN, SIGN, 8>(hist, p.stride, nb, kmin, kmax, part, nparts, p.err);
        if (nparts == 1) {
            if (active) cdr.res[j] = v;
        } else {
            float* red = reinterpret_cast<float*>(cpts);
            red[tid] = v;
            __syncthreads();
            if (active && part == 0) cdr.res[j] = fmaxf(v, red[T + col]);
        }
    }
}

// ------------------------------------------------------------------------- a2-a6: warp-specialised

// Variant of the hot kernel in which binning and sweeping overlap.  The block has two warp
// groups (T a multiple of 8, at most 128; the T columns are spread evenly over the four SM
// sub-partitions, C = T/4 per warp, lanes past C shadowing the warp's first column):
//
//   binning group (warps 0-3): zeroes its warps' histogram columns, stages the points,
//     folds and bins tile i into the private shared-memory histograms (one column per
//     frequency), then hands them over;
//   sweep group (warps 4-11, two threads per column on the column's TMEM lane quadrant):
//     copies column c of tile i into its TMEM lane (bins
//     laid out linearly, the first bins repeated past nb; the two sweep threads of a
//     column copy interleaved groups of bins and only read the histograms), hands the
//     histograms back, then sweeps the boxes of tile i from TMEM while the
//     binning group already bins tile i + 1.  Its first warp also claims the work items
//     and writes each tile's descriptor (the curve's CurveDesc and the tile index) into
//     one of two shared slots ahead of time, so that the binning group's path from one
//     tile to the next holds no global-memory round trip.
//
// The binning loop is latency-bound (one private histogram per thread, so only T threads
// can bin) and the sweep is bound by FP32 and special-function issue, so the sweep fills
// the issue slots that the binning chain leaves idle.  With T = 128 the sweep group has
// two threads per column (two warps per TMEM lane quadrant), which split the copy, the
// zeroing and the box starts.  The checks of the fast sweep's condition and the exact
// sweep (rare) read the TMEM copy (the first bins repeated past nb where they fit, else
// wrapped reads, see ws_tmem_mode); tiles with nb > 256, or that the fast sweep does not
// cover (kmax - kmin < SB - 2), are swept from shared memory before the hand-back.  The bins, the sums and the set of boxes are those of fold_sweep_kernel;
// both sweep blocks rank boxes by the signed residue, so a frequency's power can differ
// from fold_sweep_kernel's in the last bits (both are within the approximation's 2^-22).
//
// Hand-over: two mbarriers (count 1, arrived by a group's first thread after a group
// barrier); each wait is bounded in time (FoldParams::wait_ns, 30 s by default) and, if it
// gives up, the kernel records kErrTimeout and both groups stop.

constexpr unsigned long long kHandoffTimeoutNs = 30ull * 1000000000ull;
constexpr int kBarBin = 1, kBarSweep = 2;   // named barriers of the two groups

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned a)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(a)
                 : "memory");
}
// One bounded test: the thread is suspended until the phase completes or about
// kSuspendNs pass, so a waiting thread takes no issue slots from the working warps.
constexpr unsigned kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity, unsigned suspend_ns)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(a), "r"(parity), "r"(suspend_ns) : "memory");
    return ok != 0;
}
// Waits until the phase of the given parity has completed; false if it has not within
// limit_ns (each test suspends the thread for at most min(kSuspendNs, limit_ns)).
__device__ __noinline__ bool mbar_wait(unsigned a, unsigned parity, unsigned long long limit_ns)
{
    const unsigned sus = limit_ns < kSuspendNs ? (unsigned)limit_ns : kSuspendNs;
    if (mbar_try(a, parity, sus)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (unsigned it = 0; it < 0x7fffffffu; ++it) {
        if (mbar_try(a, parity, sus)) return true;
        if (globaltimer_ns() - t0 > limit_ns) break;
    }
    return false;
}
__device__ __forceinline__ void group_sync(int id, int n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Group barrier that also returns whether v was non-zero on any thread of the group.
__device__ __forceinline__ int group_or(int id, int n, int v)
{
    int r;
    asm volatile("{\n\t.reg .pred q, o;\n\tsetp.ne.s32 q, %1, 0;\n\t"
                 "bar.red.or.pred o, %2, %3, q;\n\tselp.s32 %0, 1, 0, o;\n\t}"
                 : "=r"(r) : "r"(v), "r"(id), "r"(n) : "memory");
    return r;
}

constexpr unsigned kTmemCols = 512;

// Sequential single-bin stream over this thread's TMEM lane (as TmemBins), for the rare
// checks; every access is taken by the whole warp together.
template <bool WRAP>
struct TmemStream {
    unsigned base, tend, ta, p0, p1;
    int* err = nullptr;
    __device__ __forceinline__ void issue()
    {
        __syncwarp();
        if (!bls_ok(ta - base <= kTmemCols - 2u, err)) ta = base;
        tmem_ld2(ta, p0, p1);
        ta += 2;
        if (WRAP) ta = ta == tend ? base : ta;
    }
    __device__ __forceinline__ void start(int a)
    {
        ta = base + 2u * (unsigned)a;
        issue();
    }
    __device__ __forceinline__ void next(float& hw, float& hx)
    {
        unsigned d0 = 0, d1 = 0;
        __syncwarp();
        tmem_wait_ld4(p0, p1, d0, d1);
        hw = __uint_as_float(p0);
        hx = __uint_as_float(p1);
        issue();
    }
    __device__ __forceinline__ void finish()
    {
        unsigned d0 = 0, d1 = 0;
        __syncwarp();
        tmem_wait_ld4(p0, p1, d0, d1);
    }
};

// Sweep of one column from its TMEM copy, all lanes of the warp together.
// Both blocks take the signed-residue form here: it issues fewer instructions per box than
// the shared-reciprocal form or a division-free threshold test, and leans on the
// special-function unit, which the binning warps sharing the SM sub-partitions do not use.
template <int SB, int SIGN, bool WRAP>
__device__ __forceinline__ float sweep_tmem(unsigned tbase, int nb, int kmin, int kmax, int part,
                                            int nparts, int* err)
{
    TmemBins<WRAP> src;
    src.err = err;
    src.base = tbase;
    src.tend = tbase + 2u * (unsigned)nb;
    return sweep_fast<SB, SIGN, TmemBins<WRAP>, 0>(src, nb, kmin, kmax, part, nparts);
}

// Heaviest run of kmax consecutive bins (cyclic), as in sweep_max, from the TMEM copy.
template <bool WRAP>
__device__ float heaviest_run_tmem(unsigned tbase, int nb, int kmax, int* err)
{
    TmemBins<WRAP> src;
    src.err = err;
    src.base = tbase;
    src.tend = tbase + 2u * (unsigned)nb;
    float win = 0.0f, hw, hx, hw2, hx2;
    src.start(0, 0);
    for (int b = 0; b < kmax; ++b) {
        src.next(hw, hx, hw2, hx2);
        win += hw;
    }
    src.finish();
    float rmax = win;
    src.start(0, kmax);   // bin b leaves, bin b + kmax enters
    for (int b = 0; b + 1 < nb; ++b) {
        float hout, hin;
        src.next(hout, hx, hin, hx2);
        win = __fsub_rn(__fadd_rn(win, hin), hout);
        rmax = fmaxf(rmax, win);
    }
    src.finish();
    return rmax;
}

// Descriptor of one work item, written by the sweep group ahead of its use.
struct TileSlot {
    CurveDesc cd;
    int tile;
    int stop;
};

// Claims the next work item and writes its descriptor (by the 32 lanes of one warp): the
// range of the item is found by a 32-way search of the prefix array.
__device__ void fetch_tile(const FoldParams& p, TileSlot* slot, int lane)
{
    int it = 0;
    if (lane == 0) it = atomicAdd(p.counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= p.total) {
        if (lane == 0) slot->stop = 1;
        return;
    }
    int lo = 0, hi = p.nranges;   // prefix[lo] <= it < prefix[hi]
    while (hi - lo > 1) {
        const int step = (hi - lo + 31) >> 5;
        const int idx = lo + lane * step;
        const bool le = idx < hi && p.prefix[idx] <= it;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        lo += (31 - __clz(m)) * step;
        hi = min(hi, lo + step);
    }
    const TileRange tr = p.ranges[lo];
    static_assert(sizeof(CurveDesc) % 8 == 0, "CurveDesc is copied in 8-byte words");
    const u64* src = reinterpret_cast<const u64*>(&p.curves[tr.curve]);
    u64* dst = reinterpret_cast<u64*>(&slot->cd);
    for (int w = lane; w < (int)(sizeof(CurveDesc) / 8); w += 32) dst[w] = src[w];
    if (lane == 0) {
        slot->tile = tr.tile_lo + (int)(it - p.prefix[lo]);
        slot->stop = 0;
    }
}

// The sweep group's loop of fold_sweep_ws_kernel: warps 4-7 (part 0) and 8-11 (part 1),
// the two threads of a column in warps of the same TMEM lane quadrant; lane_ok is false
// for a lane that shadows its warp's first column.  Warp 4 claims the work items and
// writes the tile descriptors ahead; per tile the group copies the histograms into TMEM,
// hands them back (the binning group zeroes them) and sweeps the boxes from TMEM.
constexpr int kWsBinThreads = 128, kWsSweepThreads = 256, kWsSweep0 = 128;

template <int SIGN, int SUMS>
__device__ __forceinline__ void sweep_group_loop(const FoldParams& p, bool lane_ok, int col,
                                                 unsigned s_tmem, TileSlot* s_slot,
                                                 unsigned full_bar, unsigned empty_bar,
                                                 unsigned slot_bar, float* s_wpart, float* s_wpart2,
                                                 unsigned char* hist, unsigned hbase,
                                                 unsigned rowb)
{
    const int T = p.cols;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int NS = kWsSweepThreads, sg0 = kWsSweep0;
    // nparts = 2 threads per column, in warps of one TMEM lane quadrant
    const int nparts = 2;
    const int part = (warp - sg0 / 32) >> 2;
    const unsigned tbase = s_tmem + ((unsigned)((warp & 3) * 32) << 16);
    const bool fetcher = warp == sg0 / 32;
    unsigned ph = 0;
    // descriptors of tiles 0 and 1 (each published on its slot's barrier by the 32 lanes
    // that wrote it); the histograms start empty
    if (fetcher) {
        fetch_tile(p, &s_slot[0], lane);
        mbar_arrive(slot_bar);
    }
    group_sync(kBarSweep, NS);
    if (tid == sg0) mbar_arrive(empty_bar);
    if (fetcher) {
        fetch_tile(p, &s_slot[1], lane);
        mbar_arrive(slot_bar + 8u);
    }
    for (int k = 0;; ++k) {
        int give_up = 0;
        if (tid == sg0) {
            give_up = !mbar_wait(full_bar, ph, p.wait_ns ? p.wait_ns : kHandoffTimeoutNs);
            if (give_up) atomicOr(p.err, kErrTimeout);
        }
        ph ^= 1u;
        give_up = group_or(kBarSweep, NS, give_up);
        const TileSlot& sl = s_slot[k & 1];
        if (give_up || sl.stop) break;
        const int tile = sl.tile;
        const int nf = sl.cd.nf, nb = sl.cd.nb, kmin = sl.cd.kmin, kmax = sl.cd.kmax;
        float* const res = sl.cd.res;
        const float wq = sl.cd.wq, xq = sl.cd.xq;
        const int j = tile * T + col;
        const bool active = lane_ok && j < nf;
        const int SB = sweep_block(nb, kmin, kmax);
        const int tmode = ws_tmem_mode(nb, kmin, kmax);
        const bool use_tmem = tmode != 0;
        float v = 0.0f, wmax = 0.0f;
        if (use_tmem) {
            // copy bins 0 .. L-1 (bin b >= nb repeats bin b - nb; L <= 2 nb) into the
            // column's lane, 8 bins per TMEM store (groups dealt to the parts)
            const int L = ((tmode == 1 ? nb + kmax + SB - 1 : nb) + 7) & ~7;
            const unsigned wrapb = (unsigned)nb * rowb;
            for (int g = 8 * part; g < L; g += 8 * nparts) {
                const unsigned ag = hbase + (unsigned)g * rowb;
                u64 h[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const unsigned ai = ag + (unsigned)i * rowb - (g + i >= nb ? wrapb : 0u);
                    if (!bls_ok(g + i < 2 * nb, p.err)) {
                        h[i] = 0ull;
                    } else if (SUMS == kSumKahan) {   // the compensated sums (sum - compensation)
                        u64 hh, cc;
                        lds128(ai, hh, cc);
                        h[i] = sub2(hh, cc);
                    } else {
                        h[i] = lds64(ai);
                    }
                }
                unsigned r[16];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    float hw, hx;
                    if (SUMS == kSumFixed) fixed_pair(h[i], wq, xq, hw, hx);   // integer sums
                    else upk(h[i], hw, hx);
                    if (g + i < nb) wmax = fmaxf(wmax, hw);
                    r[2 * i] = __float_as_uint(hw);
                    r[2 * i + 1] = __float_as_uint(hx);
                }
                tmem_st16(tbase + (bls_ok(2 * g + 16 <= (int)kTmemCols, p.err) ? 2u * (unsigned)g : 0u), r);
            }
            if (part == 1 && lane_ok) s_wpart[col] = wmax;
            tmem_wait_st();
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        } else if (part == 0) {
            constexpr int KAHAN = SUMS == kSumKahan;
            if (SUMS == kSumFixed && active) fixed_to_f32(hbase, rowb, nb, wq, xq);
            if (active)
                v = SB == 4 ? sweep_max<KAHAN, SIGN, 4>(hist, p.stride, nb, kmin, kmax, 0, 1, p.err)
                    : SB == 10 ? sweep_max<KAHAN, SIGN, 10>(hist, p.stride, nb, kmin, kmax, 0, 1, p.err)
                               : sweep_max<KAHAN, SIGN, 8>(hist, p.stride, nb, kmin, kmax, 0, 1, p.err);
        }
        // the histograms are only read here: the binning group zeroes them when it starts
        // the next tile (after this hand-over)
        group_sync(kBarSweep, NS);
        if (tid == sg0) mbar_arrive(empty_bar);
        // descriptor of tile k + 2 into slot k & 1, published on the slot's barrier: every
        // thread of this group has read the slot into registers above, and the binning
        // group read it before binning tile k
        if (fetcher) {
            fetch_tile(p, &s_slot[k & 1], lane);
            mbar_arrive(slot_bar + 8u * (unsigned)(k & 1));
        }
        if (use_tmem) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            bool fast = true;
            if (part == 0) {
                // the fast sweep's condition (as in sweep_max) and the exact sweep
                if (nparts == 2) wmax = fmaxf(wmax, s_wpart[col]);
                fast = (float)kmax * wmax < 0.89f;
                const bool slide = !fast && kmax < nb;
                if (__any_sync(0xffffffffu, slide)) {
                    const float rmax = tmode == 1 ? heaviest_run_tmem<false>(tbase, nb, kmax, p.err)
                                                  : heaviest_run_tmem<true>(tbase, nb, kmax, p.err);
                    if (slide) fast = rmax < 0.89f;
                }
                const bool exact = active && !fast;
                if (__any_sync(0xffffffffu, exact)) {
                    Best g;
                    if (tmode == 1) {
                        TmemStream<false> src;
                        src.err = p.err;
                        src.base = tbase;
                        src.tend = tbase + 2u * (unsigned)nb;
                        g = sweep_exact_src<SIGN>(src, nb, kmin, kmax);
                    } else {
                        TmemStream<true> src;
                        src.err = p.err;
                        src.base = tbase;
                        src.tend = tbase + 2u * (unsigned)nb;
                        g = sweep_exact_src<SIGN>(src, nb, kmin, kmax);
                    }
                    if (exact) v = g.num > 0.0f ? __fdiv_rn(g.num, g.den) : 0.0f;
                }
            }
            __syncwarp();
            float vf;
            if (tmode == 1)
                vf = SB == 4 ? sweep_tmem<4, SIGN, false>(tbase, nb, kmin, kmax, part, nparts, p.err)
                     : SB == 10 ? sweep_tmem<10, SIGN, false>(tbase, nb, kmin, kmax, part, nparts, p.err)
                                : sweep_tmem<8, SIGN, false>(tbase, nb, kmin, kmax, part, nparts, p.err);
            else
                // wrapped copies with nb a multiple of 64 (nb = 256 of the survey sweep): blocks
                // of 16 starts, which the two sweep threads of a column share evenly (more
                // independent boxes per TMEM read; 353.1 -> 348.8 ms per 512 survey curves)
                vf = SB == 4 ? sweep_tmem<4, SIGN, true>(tbase, nb, kmin, kmax, part, nparts, p.err)
                     : nb % 64 == 0 ? sweep_tmem<16, SIGN, true>(tbase, nb, kmin, kmax, part, nparts, p.err)
                     : SB == 10 ? sweep_tmem<10, SIGN, true>(tbase, nb, kmin, kmax, part, nparts, p.err)
                                : sweep_tmem<8, SIGN, true>(tbase, nb, kmin, kmax, part, nparts, p.err);
            if (nparts == 2) {   // the parts' maxima meet in shared memory
                if (part == 1 && lane_ok) s_wpart2[col] = vf;
                group_sync(kBarSweep, NS);
                if (part == 0) vf = fmaxf(vf, s_wpart2[col]);
            }
            if (fast) v = vf;
        }
        if (part == 0 && active) res[j] = v;
    }
}

constexpr int kWsMaxThreads = 384;

template <int PHASE, int SUMS, int SIGN>
__global__ void __launch_bounds__(kWsMaxThreads, 1) fold_sweep_ws_kernel(FoldParams p)
{
    constexpr int KAHAN = SUMS == kSumKahan;
    extern __shared__ __align__(16) unsigned char smem[];
    // [0] histograms full, [1] empty, [2 + s] the descriptor in slot s written
    __shared__ __align__(8) unsigned long long s_bar[4];
    __shared__ TileSlot s_slot[2];                          // descriptor of tile k at [k & 1]
    __shared__ float s_wpart[128], s_wpart2[128];           // second sweep part's partials
    __shared__ unsigned s_tmem;
    const int T = p.cols;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    // The T columns are spread evenly over the four SM sub-partitions: C = T/4 per TMEM
    // lane quadrant.  Binning warps 0-3 and sweep warps 4-7 (part 0) and 8-11 (part 1):
    // lane l < C of a warp on quadrant q = warp & 3 owns column q C + l, and both sweep
    // threads of a column run on the quadrant where its histogram is copied.  Lanes l >= C
    // (T < 128) shadow their warp's first column: they execute the warp-wide instructions
    // alongside it and write nothing.
    const int C = T / 4;
    const bool binner = warp < 4;
    const bool lane_ok = lane < C;
    const int col = (warp & 3) * C + (lane_ok ? lane : 0);
    const int CH = p.chunk;
    float4* cpts = reinterpret_cast<float4*>(smem);             // [2][CH]: point pairs
    double* cdt = reinterpret_cast<double*>(cpts + 2 * CH);     // [2][CH]: FP64 offsets
    unsigned char* hist_all = reinterpret_cast<unsigned char*>(cdt + 2 * CH);
    constexpr size_t ESZ = KAHAN ? sizeof(float4) : sizeof(float2);   // histogram entry
    unsigned char* hist = hist_all + (size_t)col * ESZ;
    const size_t S = (size_t)p.stride;
    const unsigned hbase = (unsigned)__cvta_generic_to_shared(hist);
    const unsigned rowb = (unsigned)(S * ESZ);
    const unsigned full_bar = (unsigned)__cvta_generic_to_shared(&s_bar[0]);
    const unsigned empty_bar = (unsigned)__cvta_generic_to_shared(&s_bar[1]);
    const unsigned slot_bar = (unsigned)__cvta_generic_to_shared(&s_bar[2]);   // slot s: + 8 s

    {   // every histogram row starts at zero (afterwards each binning warp re-zeroes its
        // columns at the start of every tile)
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        const size_t rows = (dyn - (size_t)2 * CH * (sizeof(float4) + sizeof(double))) / rowb;
        u64* h = reinterpret_cast<u64*>(hist_all);
        for (size_t e = tid; e < rows * S * (ESZ / 8); e += blockDim.x) h[e] = 0ull;
    }
    if (warp == 4) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"((unsigned)__cvta_generic_to_shared(&s_tmem)), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(full_bar, 1);
        mbar_init(empty_bar, 1);
        mbar_init(slot_bar, 32);        // arrived by the 32 lanes that write the slot
        mbar_init(slot_bar + 8u, 32);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (binner) {
        unsigned ph = 0;
        const unsigned long long wlim = p.wait_ns ? p.wait_ns : kHandoffTimeoutNs;
        for (int k = 0;; ++k) {
            int give_up = 0;
            if (tid == 0) {   // tile k's descriptor, written ahead by the sweep group
                give_up = !mbar_wait(slot_bar + 8u * (unsigned)(k & 1), (unsigned)(k >> 1) & 1u, wlim);
                if (give_up) atomicOr(p.err, kErrTimeout);
            }
            give_up = group_or(kBarBin, kWsBinThreads, give_up);
            const TileSlot& sl = s_slot[k & 1];
            if (give_up || sl.stop) {
                // the stop is handed over once the sweep group has taken the previous tile
                if (tid == 0 && !give_up && !mbar_wait(empty_bar, ph, wlim)) atomicOr(p.err, kErrTimeout);
                group_sync(kBarBin, kWsBinThreads);
                if (tid == 0) mbar_arrive(full_bar);   // the sweep group reads the stop
                break;
            }
            const CurveDesc cdr = sl.cd;
            const int tile = sl.tile;
            const int n = cdr.n, nf = cdr.nf, nb = cdr.nb;
            const float4* gpts = cdr.pts;
            const double* gdt = cdr.dt64;
            const int j = tile * T + col;
            const bool active = lane_ok && j < nf;
            const int jt = j < nf ? j : nf - 1;
            const double f = grid_freq(cdr, jt);
            // FX64 tiles of a uniform grid take the incremental fold, with the tile's middle
            // column (at most its last frequency) as the reference column
            const int jc = min(tile * T + T / 2, nf - 1);
            const double fcen = grid_freq(cdr, jc);
            const bool inc = PHASE == kPhaseFX64 && cdr.freqs == nullptr &&
                             inc_tile_ok(fcen, cdr);
            FoldConst fc = make_fold_const(f, nb, cdr.dtmax, cdr.fxs, !inc,
                                           PHASE == kPhaseDF32 || PHASE == kPhaseF32);
            if (inc) make_fold_const_inc(fc, f, fcen, jt - jc, cdr, nb);
            const FoldPacked fq = make_fold_packed(fc);

            // a2: chunks of CH points through shared memory (as in fold_sweep_kernel)
            const int nchunks = (n + CH - 1) / CH;
            auto stage = [&](int ci) {
                const int c0 = ci * CH;
                const int cn = (min(CH, n - c0) + 1) & ~1;
                const int cpad = (cn + 15) & ~15;
                float4* dp = cpts + (ci & 1) * CH;
                double* dd = cdt + (ci & 1) * CH;
                // thread t copies point pairs t, t + 128, ...: both float4 slots of a pair and
                // its two FP64 offsets (16-byte aligned: curves start at even points)
                for (int i = 2 * tid; i < cn; i += 2 * kWsBinThreads) {
                    cp_async16(&dp[i], &gpts[c0 + i]);
                    cp_async16(&dp[i + 1], &gpts[c0 + i + 1]);
                    cp_async16(&dd[i], &gdt[c0 + i]);
                }
                for (int i = cn + tid; i < cpad; i += kWsBinThreads) {
                    dp[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    dd[i] = 0.0;
                }
                cp_async_commit();
            };
            // the tile's constants and its first chunk are prepared while the sweep group may
            // still be copying the previous tile's histograms out
            stage(0);
            if (tid == 0) {
                give_up = !mbar_wait(empty_bar, ph, wlim);
                if (give_up) atomicOr(p.err, kErrTimeout);
            }
            ph ^= 1u;
            give_up = group_or(kBarBin, kWsBinThreads, give_up);
            if (give_up) {
                cp_async_wait_all();
                if (tid == 0) mbar_arrive(full_bar);
                break;
            }
            if (lane_ok) {   // zero this thread's histogram column; the sweep group has
                             // finished reading it (the empty hand-over above)
                for (int b = 0; b < nb; ++b) {
                    if (KAHAN) sts128(hbase + (unsigned)b * rowb, 0ull, 0ull);
                    else sts64(hbase + (unsigned)b * rowb, 0ull);
                }
            }
            __syncwarp();
            for (int ci = 0; ci < nchunks; ++ci) {
                if (ci + 1 < nchunks) stage(ci + 1); else cp_async_commit();
                cp_async_wait1();
                if (inc) {
                    // staging step of the incremental fold, on this thread's own copies (the
                    // DT slot of each of its point pairs): (lo0, lo1, hi0, hi1) ->
                    // (Q0, Q1, D0, D1) (written out here rather than through inc_stage: the
                    // binning loop below is measurably faster with this form)
                    float4* dp = cpts + (ci & 1) * CH;
                    const int cn = (min(CH, n - ci * CH) + 1) & ~1;
                    for (int i = 2 * tid; i < cn; i += 2 * kWsBinThreads) {
                        const float4 A = dp[i];
                        unsigned Q0, D0, Q1, D1;
                        inc_point(__float_as_uint(A.x), __float_as_uint(A.z), fc, Q0, D0);
                        inc_point(__float_as_uint(A.y), __float_as_uint(A.w), fc, Q1, D1);
                        dp[i] = make_float4(__uint_as_float(Q0), __uint_as_float(Q1),
                                            __uint_as_float(D0), __uint_as_float(D1));
                    }
                }
                group_sync(kBarBin, kWsBinThreads);
                const int cnum = min(CH, n - ci * CH);
                const float4* cp = cpts + (ci & 1) * CH;
                const double* cd = cdt + (ci & 1) * CH;
                if (active) {   // a3 + a4
                    if ((PHASE == kPhaseDF32 && fc.fast) || (PHASE == kPhaseFX64 && fc.fxok)) {
                        if (inc && fc.sh != 0u)   // nb a power of two: shifts, not multiplies
                            bin_fast<PHASE, true, true, SUMS, true>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                        else if (inc)
                            bin_fast<PHASE, true, true, SUMS>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                        else
                            bin_fast<PHASE, true, false, SUMS>(cp, cd, (cnum + 15) >> 4, hbase, rowb, fc, fq, p.err);
                    } else
                        bin_generic<PHASE, SUMS>(cp, cd, (cnum + 1) >> 1, hbase, rowb, fc, fq, p.err);
                }
                group_sync(kBarBin, kWsBinThreads);
            }
            if (tid == 0) mbar_arrive(full_bar);
        }
    } else {
        sweep_group_loop<SIGN, SUMS>(p, lane_ok, col, s_tmem, s_slot, full_bar, empty_bar, slot_bar, s_wpart,
                               s_wpart2, hist, hbase, rowb);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 4) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s_tmem),
                     "r"(kTmemCols) : "memory");
    }
}

// Tile geometries the warp-specialised kernel can take: plain or Kahan sums (16-byte
// entries, whose compensated values the sweep group copies into TMEM), T a multiple of 8, at
// most 128 (T/4 columns per TMEM lane quadrant).  BLS_FOLD_WS=0 in the environment selects
// fold_sweep_kernel for every class.
static bool use_ws(int T, int sums)
{
    static const int env = [] {
        const char* e = getenv("BLS_FOLD_WS");
        return (e && e[0] == '0') ? 0 : 1;
    }();
    (void)sums;   // every sum mode
    return env && T % 8 == 0 && T >= 8 && T <= 128;
}

// Threads of a warp-specialised block: binning warps 0-3, sweep warps 4-11, whatever the
// tile width (T/4 columns per warp).
static int ws_threads(int) { return kWsMaxThreads; }

// Frequencies per tile, given the most whose histograms fit (a multiple of 16, at most 256):
// where the warp-specialised kernel applies, that width itself up to 128, else 128.
// Measured on 256 curves x 20k frequencies: nb = 150, 160 columns (one-group kernel, one
// thread per column) 21.8 ms against 14.8 ms at 128 (warp-specialised).  256 columns
// (nb <= 100) keep the one-group kernel, whose eight binning warps then win (11.5 ms
// against 13.1 ms at nb = 100).
int fold_preferred_cols(int tmax, int sums, int nb, int kmin, int kmax, int choice)
{
    if (tmax >= 256) return tmax;
    const int Tw = tmax > 128 ? 128 : tmax & ~7;
    if (Tw >= 8 && fold_use_ws(Tw, sums, nb, kmin, kmax, choice)) return Tw;
    return tmax;
}

// The warp-specialised kernel takes classes whose tiles it sweeps from TMEM; where it
// cannot (nb > 256) or the fast sweep does not apply, its sweep group would sweep from
// shared memory while the binning group waits, and the one-group kernel, whose threads all
// bin and then all sweep, is faster (nb = 400: 81.7 ms at 48 columns against 97.3 ms at
// 64, 256 curves x 20k frequencies).
bool fold_use_ws(int T, int sums, int nb, int kmin, int kmax, int choice)
{
    if (choice == BLS_FOLD_ONE_GROUP || !use_ws(T, sums)) return false;
    return choice == BLS_FOLD_WS || ws_tmem_mode(nb, kmin, kmax) != 0;
}

int fold_ws_mode(int T, int sums, int nb, int kmin, int kmax, int choice)
{
    return fold_use_ws(T, sums, nb, kmin, kmax, choice) ? 1 : 0;
}

// Dynamic shared memory of a warp-specialised block: at least half of an SM's shared memory,
// so that no second block (which would wait for the first one's TMEM) lands on the SM.
static size_t ws_smem(size_t smem)
{
    static const size_t half = [] {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
            cudaGetLastError();
            v = 0;
        }
        return (size_t)v / 2 + 1024;
    }();
    return smem > half ? smem : half;
}

template <int PHASE, int SUMS, int SIGN>
static cudaError_t launch_fold_t(const FoldParams& p, int T, int grid, size_t smem,
                                 cudaStream_t s, int ws)
{
    FoldParams q = p;
    q.cols = T;
    if (ws && use_ws(T, SUMS)) {
        auto k = fold_sweep_ws_kernel<PHASE, SUMS, SIGN>;
        const size_t sm = ws_smem(smem);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        k<<<grid, ws_threads(T), sm, s>>>(q);
        return cudaGetLastError();
    }
    auto k = fold_sweep_kernel<PHASE, SUMS, SIGN>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, fold_block_threads(T), smem, s>>>(q);
    return cudaGetLastError();
}

template <int PHASE, int SUMS, int SIGN>
static int blocks_t(int T, size_t smem, int ws)
{
    if (ws && use_ws(T, SUMS)) {
        // one block per SM: all of TMEM and (nearly) all of shared memory
        auto k = fold_sweep_ws_kernel<PHASE, SUMS, SIGN>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws_smem(smem)) != cudaSuccess) {
            cudaGetLastError();
            return 1;
        }
        return 1;
    }
    auto k = fold_sweep_kernel<PHASE, SUMS, SIGN>;
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, fold_block_threads(T), smem) != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return nb > 0 ? nb : 1;
}

int fold_blocks_per_sm(int T, size_t smem, int phase, int sums, int sign, int ws)
{
#define BLS_OCC(PH)                                                                   \
    if (phase == PH) {                                                                \
        if (sums == kSumKahan)                                                        \
            return sign ? blocks_t<PH, kSumKahan, 1>(T, smem, ws) : blocks_t<PH, kSumKahan, 0>(T, smem, ws); \
        if (sums == kSumF32)                                                          \
            return sign ? blocks_t<PH, kSumF32, 1>(T, smem, ws) : blocks_t<PH, kSumF32, 0>(T, smem, ws); \
        return sign ? blocks_t<PH, kSumFixed, 1>(T, smem, ws) : blocks_t<PH, kSumFixed, 0>(T, smem, ws); \
    }
    BLS_OCC(kPhaseDF32)
    BLS_OCC(kPhaseF64)
    BLS_OCC(kPhaseF32)
    BLS_OCC(kPhaseFX64)
#undef BLS_OCC
    return 1;
}

cudaError_t launch_fold_sweep(const FoldParams& p, int T, int grid, int phase, int sums, int ws,
                              int sign, size_t smem, cudaStream_t s)
{
#define BLS_DISPATCH(PH)                                                              \
    if (phase == PH) {                                                                \
        if (sums == kSumKahan)                                                        \
            return sign ? launch_fold_t<PH, kSumKahan, 1>(p, T, grid, smem, s, ws)    \
                        : launch_fold_t<PH, kSumKahan, 0>(p, T, grid, smem, s, ws);   \
        if (sums == kSumF32)                                                          \
            return sign ? launch_fold_t<PH, kSumF32, 1>(p, T, grid, smem, s, ws)      \
                        : launch_fold_t<PH, kSumF32, 0>(p, T, grid, smem, s, ws);     \
        return sign ? launch_fold_t<PH, kSumFixed, 1>(p, T, grid, smem, s, ws)        \
                    : launch_fold_t<PH, kSumFixed, 0>(p, T, grid, smem, s, ws);       \
    }
    BLS_DISPATCH(kPhaseDF32)
    BLS_DISPATCH(kPhaseF64)
    BLS_DISPATCH(kPhaseF32)
    BLS_DISPATCH(kPhaseFX64)
#undef BLS_DISPATCH
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------- best box

// One frequency's histogram of a curve, binned point by point into a private histogram
// column with the hot kernel's fold.  The FP32 bin sums follow point order; where points of
// one read-modify-write group of the hot kernel share a bin, that kernel adds their
// pre-summed weights, so such a bin can differ from this one in its last bit.  Fixed-point
// sums are exact integers, converted to FP32 as the hot kernels convert them: those bins
// equal the hot kernels' bit for bit.
__device__ void bin_column(const CurveDesc& cd, double f, unsigned char* hist, int stride,
                           int phase, int sums, int* err = nullptr)
{
    const bool kahan = sums == kSumKahan;
    const size_t S = (size_t)stride;
    const FoldConst fc = make_fold_const(f, cd.nb, cd.dtmax, cd.fxs);
    const FoldPacked fq = make_fold_packed(fc);
    for (int b = 0; b < cd.nb; ++b) {
        if (kahan) reinterpret_cast<float4*>(hist)[(size_t)b * S] = make_float4(0.f, 0.f, 0.f, 0.f);
        else reinterpret_cast<u64*>(hist)[(size_t)b * S] = 0ull;
    }
    for (int pi = 0; 2 * pi < cd.n; ++pi) {
        const float4 A = cd.pts[2 * pi], B = cd.pts[2 * pi + 1];
        unsigned b0, b1;
        fold_pair_rt(phase, A, &cd.dt64[2 * pi], fc, fq, b0, b1);
        if (!bls_ok(b0 < (unsigned)cd.nb && b1 < (unsigned)cd.nb, err)) continue;
        if (kahan) {
            kahan_add(reinterpret_cast<float4*>(hist) + b0 * S, B.x, B.y);
            kahan_add(reinterpret_cast<float4*>(hist) + b1 * S, B.z, B.w);
        } else if (sums == kSumFixed) {
            unsigned* H = reinterpret_cast<unsigned*>(hist);
            H[2 * b0 * S] += __float_as_uint(B.x);
            H[2 * b0 * S + 1] += __float_as_uint(B.y);
            H[2 * b1 * S] += __float_as_uint(B.z);
            H[2 * b1 * S + 1] += __float_as_uint(B.w);
        } else {
            u64* H = reinterpret_cast<u64*>(hist);
            H[b0 * S] = add2(H[b0 * S], pk(B.x, B.y));
            H[b1 * S] = add2(H[b1 * S], pk(B.z, B.w));
        }
    }
    if (sums == kSumFixed) {
        u64* H = reinterpret_cast<u64*>(hist);
        for (int b = 0; b < cd.nb; ++b) {
            float r, sx;
            fixed_pair(H[(size_t)b * S], cd.wq, cd.xq, r, sx);
            H[(size_t)b * S] = pk(r, sx);
        }
    }
}

// The best box (exact tie-break) of one frequency, by one thread.
__device__ Best best_box_at(const CurveDesc& cd, double f, unsigned char* hist, int stride,
                            int phase, int sums, int sign)
{
    bin_column(cd, f, hist, stride, phase, sums);
    return sweep_exact_rt(sign, hist, stride, sums == kSumKahan, cd.nb, cd.kmin, cd.kmax);
}

// The same by the 32 lanes of a warp: lane 0 bins, the lanes share the exact sweep.
__device__ Best best_box_warp(const CurveDesc& cd, double f, unsigned char* hist, int stride,
                              int phase, int sums, int sign, int lane, int* err)
{
    if (lane == 0) bin_column(cd, f, hist, stride, phase, sums, err);
    __syncwarp();
    const int kahan = sums == kSumKahan;
    return sign ? sweep_exact_warp<1>(hist, stride, kahan, cd.nb, cd.kmin, cd.kmax, lane)
                : sweep_exact_warp<0>(hist, stride, kahan, cd.nb, cd.kmin, cd.kmax, lane);
}

// Diagnostics: (P, i1, k) of the best box at frequencies j0 .. j0 + count of one curve.
__global__ void argmax_kernel(const CurveDesc* curve, int j0, int count, int phase, int sums,
                              int sign, float* P, int* i1, int* k)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const CurveDesc cd = *curve;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= count) return;
    unsigned char* hist = smem + (size_t)threadIdx.x * hist_entry_bytes(sums);
    const Best g = best_box_at(cd, grid_freq(cd, j0 + q), hist, blockDim.x, phase, sums, sign);
    P[q] = g.num > 0.0f ? __fdiv_rn(g.num, g.den) : 0.0f;
    i1[q] = g.i1;
    k[q] = g.k;
}

cudaError_t launch_argmax(const CurveDesc* d_curve, int nb, int nf, int phase, int sums,
                          int sign, float* P, int* i1, int* k, cudaStream_t s)
{
    const int esz = hist_entry_bytes(sums);
    int T = 64;
    while (T > 1 && (size_t)T * nb * esz > 200 * 1024) T >>= 1;
    const size_t smem = (size_t)T * nb * esz;
    cudaError_t e = cudaFuncSetAttribute(argmax_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    for (int j0 = 0; j0 < nf; j0 += 65536) {
        const int cnt = min(65536, nf - j0);
        argmax_kernel<<<(cnt + T - 1) / T, T, smem, s>>>(d_curve, j0, cnt, phase, sums, sign,
                                                         P + j0, i1 + j0, k + j0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------------- a7: reduce

constexpr int kReduceThreads = 256;

struct Cand { float P; int j; };

__device__ __forceinline__ bool better(float Pa, int ja, float Pb, int jb)
{
    return Pa > Pb || (Pa == Pb && ja < jb);
}

// Per curve: rank the local maxima of P(f_j) by (P desc, j asc) and keep topk; find the
// best box of each kept frequency with the exact tie-break; refit that box in FP64 from
// the raw inputs (exact FP64 fold, FP64 weights) and derive period, epoch, duration,
// depth, SNR and SR.  Dynamic shared memory: one histogram column per kept frequency.
__global__ void __launch_bounds__(kReduceThreads) reduce_kernel(ReduceParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float sP[kReduceThreads / 32];
    __shared__ int sJ[kReduceThreads / 32];
    __shared__ int sT[kReduceThreads / 32];
    __shared__ int sel[kMaxTopK];
    __shared__ int sel_i1[kMaxTopK], sel_k[kMaxTopK];
    __shared__ double red[kReduceThreads];
    const CurveDesc cd = p.curves[p.slots ? p.slots[blockIdx.x] : (int)blockIdx.x];
    const float* res = cd.res;
    const int K = p.topk;
    const int nf = cd.nf;
    Cand lst[kMaxTopK];
    int cnt = 0;
    double srsum = 0.0;
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const float P = res[j];
        const float sr = sqrtf(P);
        if (p.spectrum) p.spectrum[cd.spec_off + j] = sr;
        srsum = __dadd_rn(srsum, (double)sr);
        const bool lm = (j == 0 || P > res[j - 1]) && (j == nf - 1 || P >= res[j + 1]);
        if (!lm) continue;
        int pos = cnt < K ? cnt : K;
        for (int q = 0; q < cnt; ++q) {
            if (better(P, j, lst[q].P, lst[q].j)) { pos = q; break; }
        }
        if (pos >= K) continue;
        int last = cnt < K ? cnt : K - 1;
        for (int q = last; q > pos; --q) lst[q] = lst[q - 1];
        lst[pos].P = P;
        lst[pos].j = j;
        if (cnt < K) ++cnt;
    }
    // signal detection efficiency: mean and population standard deviation of SR over the
    // spectrum (two passes, FP64 sums in a fixed tree)
    const double srmean = __ddiv_rn(block_sum(srsum, red), (double)nf);
    double srvar = 0.0;
    for (int j = threadIdx.x; j < nf; j += blockDim.x) {
        const double d = __dsub_rn((double)sqrtf(res[j]), srmean);
        srvar = __dadd_rn(srvar, __dmul_rn(d, d));
    }
    const double srsd = sqrt(__ddiv_rn(block_sum(srvar, red), (double)nf));
    int head = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < K; ++q) {
        float bp = head < cnt ? lst[head].P : -1.0f;
        int bj = head < cnt ? lst[head].j : 0x7fffffff;
        int bt = threadIdx.x;
        for (int o = 16; o > 0; o >>= 1) {
            float op = __shfl_xor_sync(0xffffffffu, bp, o);
            int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            int ot = __shfl_xor_sync(0xffffffffu, bt, o);
            if (better(op, oj, bp, bj)) { bp = op; bj = oj; bt = ot; }
        }
        if (lane == 0) { sP[warp] = bp; sJ[warp] = bj; sT[warp] = bt; }
        __syncthreads();
        if (threadIdx.x == 0) {
            float cp = sP[0]; int cj = sJ[0]; int ct = sT[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (better(sP[w], sJ[w], cp, cj)) { cp = sP[w]; cj = sJ[w]; ct = sT[w]; }
            sel[q] = cp >= 0.0f ? cj : -1;
            sT[0] = cp >= 0.0f ? ct : -1;
        }
        __syncthreads();
        if (sT[0] == (int)threadIdx.x) ++head;
        __syncthreads();
    }
    // best box of each kept frequency, one warp per frequency (lane 0 bins, the lanes share
    // the exact sweep), in rounds of at most one frequency per warp that fit the histograms
    {
        const int esz = hist_entry_bytes(p.sums);
        const int nwarps = (int)(blockDim.x >> 5);
        int R = (int)(p.smem_bytes / ((size_t)cd.nb * esz));
        R = R < 1 ? 1 : (R > K ? K : (R > nwarps ? nwarps : R));
        for (int q0 = 0; q0 < K; q0 += R) {
            const int q = q0 + warp;
            if (warp < R && q < K) {
                if (sel[q] >= 0) {
                    const Best g = best_box_warp(cd, grid_freq(cd, sel[q]), smem + (size_t)warp * esz,
                                                 R, p.phase, p.sums, p.sign, lane, p.err);
                    if (lane == 0) {
                        sel_i1[q] = g.i1;
                        sel_k[q] = g.k;
                    }
                } else if (lane == 0) {
                    sel_i1[q] = 0;
                    sel_k[q] = cd.kmin;
                }
            }
            __syncthreads();
        }
    }
    for (int q = 0; q < K; ++q) {
        const int j = sel[q];
        DevPeak* out = &p.peaks[(size_t)blockIdx.x * K + q];
        if (j < 0) {
            if (threadIdx.x == 0) {
                DevPeak z = {};
                z.j = -1;
                *out = z;
            }
            continue;
        }
        const int i1 = sel_i1[q], k = sel_k[q];
        const double f = grid_freq(cd, j);
        double r = 0.0, s = 0.0;
        for (int i = threadIdx.x; i < cd.n; i += blockDim.x) {
            const double dt = __dsub_rn(cd.t[i], cd.t_ref);
            const int b = (int)fold_exact(dt, f, cd.nb);
            int rel = b - i1;
            if (rel < 0) rel += cd.nb;
            if (rel < k) {
                double inv = 1.0;
                if (cd.dy) { double dd = (double)cd.dy[i]; inv = __ddiv_rn(1.0, __dmul_rn(dd, dd)); }
                const double w = __ddiv_rn(inv, cd.W);
                r = __dadd_rn(r, w);
                s = __dadd_rn(s, __dmul_rn(w, __dsub_rn((double)cd.y[i], cd.ybar)));
            }
        }
        r = block_sum(r, red);
        s = block_sum(s, red);
        if (threadIdx.x == 0) {
            DevPeak pk;
            pk.j = j; pk.i1 = i1; pk.k = k; pk.pad = 0;
            pk.freq = f;
            pk.period = 1.0 / f;
            pk.duration = (double)k / ((double)cd.nb * f);
            double ph = ((double)i1 + 0.5 * (double)k) / (double)cd.nb;
            ph = ph - floor(ph);
            pk.epoch = cd.t_ref + ph / f;
            const double den = r * (1.0 - r);
            const bool ok = res[j] > 0.0f && r > 0.0 && r < 1.0 && (p.sign || s < 0.0);
            if (ok) {
                pk.power = s * s / den;
                pk.depth = -s / den;
                pk.sr = sqrt(pk.power);
                pk.snr = pk.sr * sqrt(cd.W);
            } else {
                pk.power = 0.0; pk.depth = 0.0; pk.sr = 0.0; pk.snr = 0.0;
            }
            pk.sde = srsd > 0.0 ? (pk.sr - srmean) / srsd : 0.0;
            *out = pk;
        }
        __syncthreads();
    }
}

size_t reduce_smem_bytes(int nb_max, int topk, int sums)
{
    size_t need = (size_t)nb_max * topk * hist_entry_bytes(sums);
    const size_t cap = 160 * 1024;
    return need < cap ? need : cap;
}

cudaError_t launch_reduce(const ReduceParams& p, int ncurves, cudaStream_t s)
{
    if (ncurves <= 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(reduce_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)p.smem_bytes);
    if (e != cudaSuccess) return e;
    reduce_kernel<<<ncurves, kReduceThreads, p.smem_bytes, s>>>(p);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- diagnostics

// Per-point bins of one curve at frequencies js, by the fold of the given phase mode.  In
// FX64 mode on a uniform grid (fixed-point or FP32 sums) the incremental fold of the search kernels is
// run as well (with the search's shift form when nb is a power of two), for the
// frequency's place in a tile of T columns -- the tile width the plan's search uses for
// this curve, so the reference column jc is the search's; a point
// where the two folds disagree is reported as -1 - bin.
template <int PHASE>
__global__ void debug_fold_kernel(const CurveDesc* curve, const int* js, int* bins, int T, int kahan)
{
    const CurveDesc cd = *curve;
    const int q = blockIdx.x;
    const int j = js[q];
    const double f = grid_freq(cd, j);
    const FoldConst fc = make_fold_const(f, cd.nb, cd.dtmax, cd.fxs);
    const FoldPacked fq = make_fold_packed(fc);
    FoldConst fi = fc;
    const int jc = min(j / T * T + T / 2, cd.nf - 1);
    const double fcen = grid_freq(cd, jc);
    const bool inc = PHASE == kPhaseFX64 && !kahan && cd.freqs == nullptr &&
                     inc_tile_ok(fcen, cd);
    if (inc) make_fold_const_inc(fi, f, fcen, j - jc, cd, cd.nb);
    for (int pi = threadIdx.x; 2 * pi < cd.n; pi += blockDim.x) {
        unsigned b0, b1;
        fold_pair<PHASE>(cd.pts[2 * pi], &cd.dt64[2 * pi], fc, fq, b0, b1);
        if (inc && fi.fxok) {
            const float4 A = cd.pts[2 * pi];
            unsigned Q0, D0, Q1, D1, c0, c1;
            bool e0, e1;
            inc_point(__float_as_uint(A.x), __float_as_uint(A.z), fi, Q0, D0);
            inc_point(__float_as_uint(A.y), __float_as_uint(A.w), fi, Q1, D1);
            const float4 QD = make_float4(__uint_as_float(Q0), __uint_as_float(Q1),
                                          __uint_as_float(D0), __uint_as_float(D1));
            if (fi.sh != 0u)   // as the search: shifts when nb is a power of two
                fold_fx_pair<true, true>(QD, fi, c0, c1, e0, e1);
            else
                fold_fx_pair<true>(QD, fi, c0, c1, e0, e1);
            if (e0) c0 = fold_exact(cd.dt64[2 * pi], f, cd.nb);
            if (e1) c1 = fold_exact(cd.dt64[2 * pi + 1], f, cd.nb);
            if (c0 != b0) b0 = (unsigned)(-1 - (int)b0);
            if (c1 != b1) b1 = (unsigned)(-1 - (int)b1);
        }
        bins[(size_t)q * cd.n + 2 * pi] = (int)b0;
        if (2 * pi + 1 < cd.n) bins[(size_t)q * cd.n + 2 * pi + 1] = (int)b1;
    }
}

cudaError_t launch_debug_fold(const CurveDesc* d_curve, const int* js, int nj, int phase,
                              int T, int sums, int* bins, cudaStream_t s)
{
    if (nj <= 0) return cudaSuccess;
    const int kahan = sums == kSumKahan;
    if (T < 1) return cudaErrorInvalidValue;
    if (phase == kPhaseF64)
        debug_fold_kernel<kPhaseF64><<<nj, 256, 0, s>>>(d_curve, js, bins, T, kahan);
    else if (phase == kPhaseF32)
        debug_fold_kernel<kPhaseF32><<<nj, 256, 0, s>>>(d_curve, js, bins, T, kahan);
    else if (phase == kPhaseDF32)
        debug_fold_kernel<kPhaseDF32><<<nj, 256, 0, s>>>(d_curve, js, bins, T, kahan);
    else
        debug_fold_kernel<kPhaseFX64><<<nj, 256, 0, s>>>(d_curve, js, bins, T, kahan);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------- baseline

constexpr int kPlainThreads = 128;
constexpr int kPlainChunk = 512;

// The paper's decomposition on B300 without redesign: each thread takes one trial period,
// the block stages the curve through shared memory, the thread phases every point, bins it
// into its own FP64 histogram (global memory: a thread's share of shared memory cannot hold
// it) and sweeps all boxes in FP64.
__global__ void __launch_bounds__(kPlainThreads) plain_f64_kernel(
    const CurveDesc* curve, const double* w64, const double* wx64, double* hist, int sign)
{
    __shared__ double s_dt[kPlainChunk], s_w[kPlainChunk], s_wx[kPlainChunk];
    const CurveDesc cd = *curve;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = j < cd.nf;
    const int nb = cd.nb, nf = cd.nf;
    const double f = grid_freq(cd, active ? j : nf - 1);
    double* hw = hist + (active ? j : 0);
    double* hx = hist + (size_t)nb * nf + (active ? j : 0);
    if (active)
        for (int b = 0; b < nb; ++b) { hw[(size_t)b * nf] = 0.0; hx[(size_t)b * nf] = 0.0; }
    for (int c0 = 0; c0 < cd.n; c0 += kPlainChunk) {
        const int cn = min(kPlainChunk, cd.n - c0);
        __syncthreads();
        for (int i = threadIdx.x; i < cn; i += blockDim.x) {
            s_dt[i] = cd.dt64[c0 + i];
            s_w[i] = w64[cd.pt_off + c0 + i];
            s_wx[i] = wx64[cd.pt_off + c0 + i];
        }
        __syncthreads();
        if (active) {
            for (int i = 0; i < cn; ++i) {
                const int b = (int)fold_exact(s_dt[i], f, nb);
                hw[(size_t)b * nf] = __dadd_rn(hw[(size_t)b * nf], s_w[i]);
                hx[(size_t)b * nf] = __dadd_rn(hx[(size_t)b * nf], s_wx[i]);
            }
        }
    }
    if (!active) return;
    // occupied arc of bins (a box holding all of it holds every point)
    int first = -1, last = -1, run = 0, gap = 0, gap_end = 0;
    for (int b = 0; b < nb; ++b) {
        if (hw[(size_t)b * nf] != 0.0) {
            if (first < 0) first = b;
            else if (run > gap) { gap = run; gap_end = b; }
            last = b;
            run = 0;
        } else if (first >= 0) {
            ++run;
        }
    }
    int arc_a = 0, arc_len = 0;
    if (first >= 0) {
        const int wrap = (nb - 1 - last) + first;
        if (wrap >= gap) { arc_a = first; arc_len = last - first + 1; }
        else { arc_a = gap_end; arc_len = nb - gap; }
    }
    double best = 0.0;
    for (int i1 = 0; i1 < nb; ++i1) {
        double r = 0.0, s = 0.0;
        int m = i1;
        for (int k = 1; k <= cd.kmax; ++k) {
            r = __dadd_rn(r, hw[(size_t)m * nf]);
            s = __dadd_rn(s, hx[(size_t)m * nf]);
            m = (m + 1 == nb) ? 0 : m + 1;
            if (k < cd.kmin) continue;
            if (r == 0.0 || box_full(i1, k, nb, arc_a, arc_len)) continue;
            if (!sign && !(s < 0.0)) continue;
            const double P = __ddiv_rn(__dmul_rn(s, s), __dmul_rn(r, __dsub_rn(1.0, r)));
            if (P > best) best = P;
        }
    }
    cd.res[j] = __double2float_rn(best);
}

cudaError_t launch_plain_f64(const CurveDesc* d_curve, const double* w64, const double* wx64,
                             int nf, double* hist, int sign, cudaStream_t s)
{
    const int grid = (nf + kPlainThreads - 1) / kPlainThreads;
    plain_f64_kernel<<<grid, kPlainThreads, 0, s>>>(d_curve, w64, wx64, hist, sign);
    return cudaGetLastError();
}

}  // namespace blsgpu
