/*
 * The oracle's PRADMM iteration executed in single precision -- TEST
 * INFRASTRUCTURE, a tolerance reference only (never an expected value).
 *
 * This unit compiles pradmm_oracle.c unchanged with its real type set to
 * float (and -fsingle-precision-constant), so every operation of the
 * checker's own algorithm rounds to FP32.  Run from the same start, its
 * deviation from the FP64 oracle at a vertex is the error an FP32 execution
 * of Eq. (3a)-(3f) picks up there: large where the vertex's update is ill
 * conditioned (|u_i| small against its terms, cancellation in t_j - s_i),
 * small elsewhere.  The tests bound the CUDA path's FP32 error per element
 * by a multiple of it.  The system headers are included first so that only
 * the oracle's own declarations change type.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#define double float
#include "pradmm_oracle.c"
