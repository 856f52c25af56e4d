// internal.h -- entry points shared between translation units of the library
// (not part of the public C ABI).
#pragma once
#include <stddef.h>

#include "ads.h"

// Number of doubles in one interior scratch field of `sim` (padded layout).
size_t ads_internal_interior_count(const ads_sim_t *sim);

// Apply ADS_OP_* like ads_apply to device arrays `in`/`out` (full space,
// FP64), using the caller's two interior scratch fields s0, s1 (each at least
// ads_internal_interior_count doubles) instead of allocating.  The caller
// makes the simulation's device current.  Waits.
int ads_internal_apply_scratch(ads_sim_t *sim, int op, const double *in, double *out, size_t count, double *s0,
                               double *s1);

// CUDA device ordinal of the simulation.
int ads_internal_sim_device(const ads_sim_t *sim);

// Record an error message for ads_last_error() and return code.
int ads_internal_fail(int code, const char *msg);
