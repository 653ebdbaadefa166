// Generated by gen_erfc_poly.py: erfcx(x) ~ sum_k Q[k] t^k, t = 1/(2+x).
#pragma once
// x in [0, 5], degree 8: max relative error 4.04e-08 (FP64 fit), 2.73e-07 (FP32 Horner).
#define SE_ERFC_DEG5 8
__device__ __constant__ const float ERFC_Q5[9] = {
    -3.140412841e-04f,
    5.753442071e-01f,
    9.572063143e-01f,
    3.456189718e+00f,
    -5.065450449e+00f,
    2.883738475e+01f,
    -5.120080445e+01f,
    3.827199462e+01f,
    -1.081557466e+01f,
};
// x in [0, 8], degree 10: max relative error 3.02e-09 (FP64 fit), 2.74e-07 (FP32 Horner).
#define SE_ERFC_DEG8 10
__device__ __constant__ const float ERFC_Q8[11] = {
    1.577578176e-05f,
    5.633506249e-01f,
    1.148018439e+00f,
    1.708092791e+00f,
    5.143675653e+00f,
    -1.086777728e+01f,
    5.292300248e+01f,
    -1.434845861e+02f,
    1.912034980e+02f,
    -1.289957813e+02f,
    3.587957741e+01f,
};
