// Sweep kernels for the two-rocket game in relative coordinates (Appendix D), n = 3.
#include "dispatch.h"
#define HJG_GAME RocketsRel3
HJG_GENERIC_GAME_TU(RocketsRel3, kernels_rockets_rel3)
