// Sweep kernels for one murmuration agent's game (per-state neighbour data), n = 4.
#include "dispatch.h"
#define HJG_GAME Flock4
HJG_GENERIC_GAME_TU(Flock4, kernels_flock4)
