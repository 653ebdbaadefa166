// Generated by gen_erfc_poly.py: erfcx(x) ~ sum_k ERFC_Q[k] t^k, t = 2/(2+x), x in [0, 8].
// Max relative error of the fit 3.02e-09 (FP64), 2.74e-07 (FP32 Horner).
#pragma once
#define SE_ERFC_XMAX 8.0f
#define SE_ERFC_DEG 10
__device__ __constant__ const float ERFC_Q[11] = {
    1.577578176e-05f,
    2.816753124e-01f,
    2.870046097e-01f,
    2.135115989e-01f,
    3.214797283e-01f,
    -3.396180399e-01f,
    8.269219137e-01f,
    -1.120973329e+00f,
    7.468886640e-01f,
    -2.519448853e-01f,
    3.503864982e-02f,
};
