// Sweep kernels for the relative Dubins game (Appendix D.2), n = 3.
#include "dispatch.h"
#define HJG_GAME Dubins3
HJG_GENERIC_GAME_TU(Dubins3, kernels_dubins3)
