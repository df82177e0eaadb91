// Generated by fit_sincos.py -- do not edit.
// FP32 minimax-style polynomials on |r| <= 1.572796 (Lawson-weighted least squares).
// Polynomial error (double evaluation): sin 4.87e-09, cos 5.36e-08.
// Float32 Horner evaluation error (sampled): sin 8.25e-08, cos 1.57e-07.
#pragma once
#define GNA_SIN_C1 (-1.666665673e-01f)
#define GNA_SIN_C2 (8.333008736e-03f)
#define GNA_SIN_C3 (-1.980601664e-04f)
#define GNA_SIN_C4 (2.598767651e-06f)
#define GNA_COS_C1 (-4.999993145e-01f)
#define GNA_COS_C2 (4.166396707e-02f)
#define GNA_COS_C3 (-1.385575277e-03f)
#define GNA_COS_C4 (2.319028135e-05f)
// pi = PI_A + PI_B + PI_C; PI_A and PI_B have 12 significant bits.
#define GNA_PI_A (3.140625f)
#define GNA_PI_B (0.00096750259399414062f)
#define GNA_PI_C (1.509958025e-07f)
// pi = PI_A + PI_B2 + e2 with PI_B2 the float32 rounding of pi - PI_A, |e2| = 5.13e-12.
#define GNA_PI_B2 (9.676535847e-04f)
#define GNA_PI_E2 (5.127e-12)
#define GNA_INV_PI_F (3.183098733e-01f)
// pi = PI_DA + PI_DB + PI_DC in double; PI_DA, PI_DB have 26 significant bits.
#define GNA_PI_DA (3.1415926218032837)
#define GNA_PI_DB (3.1786509424591713e-08)
#define GNA_PI_DC (1.2246467991473532e-16)
#define GNA_INV_PI_D (0.31830988618379069)
