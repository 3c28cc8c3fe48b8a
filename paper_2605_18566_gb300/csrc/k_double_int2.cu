// Sweep kernels for the double integrator (Appendix D), n = 2.
#include "dispatch.h"
#define HJG_GAME DoubleInt2
HJG_GENERIC_GAME_TU(DoubleInt2, kernels_double_int2)
