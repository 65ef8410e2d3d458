/*
 * evfdlb_oracle_cs.c -- the oracle compiled over double complex for
 * complex-step differentiation (entry points orc_cs_*).  TEST INFRASTRUCTURE
 * ONLY, like evfdlb_oracle.c, whose arithmetic it reuses unchanged: the
 * tangent-linear map of any oracle routine is J v = Im f(x + i h v) / h.
 */
#define ORC_COMPLEX
#include "evfdlb_oracle.c"
