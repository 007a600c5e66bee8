// ff.cuh -- float-float arithmetic on the FP32 pipes: error-free
// transformations (Knuth's two-sum and two-difference, Dekker's fast two-sum
// for ordered operands, FMA product errors) and the unevaluated sums of two
// floats (about 44 significant bits) built from them.  Shared by the pair
// kernels and the sigma(x) kernel.
#pragma once

namespace lsm {

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

// Fold the low word back into the high word (Fast2Sum), so that the low word
// never grows into a running FP32 sum of its own over many additions.
__device__ __forceinline__ void renorm(float& hi, float& lo)
{
    const float s = hi + lo;
    lo = lo - (s - hi);
    hi = s;
}

__device__ __forceinline__ void two_sum_acc64(double& hi, double& lo, double x)
{
    const double s = hi + x;
    const double bp = s - hi;
    const double err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e)
{
    s = a - b;
    const float bb = s - a;
    e = (a - (s - bb)) - (b + bb);
}


// two_sum for a, b >= 0: the larger first makes Dekker's fast two-sum exact;
// the ordering runs on the ALU pipe, the sum on three FP32 additions
__device__ __forceinline__ void two_sum_nonneg(float a, float b, float& s, float& e)
{
    const float hi = fmaxf(a, b), lo = fminf(a, b);
    s = hi + lo;
    e = lo - (s - hi);
}

// ff product of (ah, al) and (bh, bl)
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& h, float& l)
{
    h = ah * bh;
    l = fmaf(ah, bh, -h) + fmaf(ah, bl, al * bh);
}
// ff sum (ah, al) + (bh, bl), renormalised
__device__ __forceinline__ void ff_add(float ah, float al, float bh, float bl, float& h, float& l)
{
    float s, e;
    two_sum(ah, bh, s, e);
    e += al + bl;
    h = s + e;
    l = e - (h - s);
}

}  // namespace lsm
