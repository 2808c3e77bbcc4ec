// int16x2 kernel instantiations: CTAs of 4 warps, launch mode 3 (SwMode).
#define CM_W 4
#define CM_MODE 3
#define CM_LAUNCH launch_sw16_w4_m3
#define CM_OCC sw16_occ_w4_m3
#include "sw16_inst.cuh"
