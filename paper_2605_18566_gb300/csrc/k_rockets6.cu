// Sweep kernels for the two-rocket planar game, n = 6.
#include "dispatch.h"
#define HJG_GAME Rockets6
HJG_GENERIC_GAME_TU(Rockets6, kernels_rockets6)
