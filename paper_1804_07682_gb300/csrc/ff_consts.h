// Generated by fit_sincos.py -- do not edit.
// FP32 minimax-style polynomials on |r| <= 1.572796 (Lawson-weighted least squares).
// Polynomial error (double evaluation): sin 2.72e-10, cos 4.40e-10.
// Float32 Horner evaluation error (sampled): sin 8.25e-08, cos 1.20e-07.
#pragma once
#define GNA_SIN_C1 (-1.666666716e-01f)
#define GNA_SIN_C2 (8.333348669e-03f)
#define GNA_SIN_C3 (-1.984277042e-04f)
#define GNA_SIN_C4 (2.760946018e-06f)
#define GNA_SIN_C5 (-2.519737485e-08f)
#define GNA_COS_C1 (-5.000000000e-01f)
#define GNA_COS_C2 (4.166665673e-02f)
#define GNA_COS_C3 (-1.388858538e-03f)
#define GNA_COS_C4 (2.477017551e-05f)
#define GNA_COS_C5 (-2.620884629e-07f)
// pi = PI_A + PI_B + PI_C; PI_A and PI_B have 12 significant bits.
#define GNA_PI_A (3.140625f)
#define GNA_PI_B (0.00096750259399414062f)
#define GNA_PI_C (1.509958025e-07f)
#define GNA_INV_PI_F (3.183098733e-01f)
// pi = PI_DA + PI_DB + PI_DC in double; PI_DA, PI_DB have 26 significant bits.
#define GNA_PI_DA (3.1415926218032837)
#define GNA_PI_DB (3.1786509424591713e-08)
#define GNA_PI_DC (1.2246467991473532e-16)
#define GNA_INV_PI_D (0.31830988618379069)
