// int16x2 kernel instantiations: CTAs of 16 warps, launch mode 3 (SwMode).
#define CM_W 16
#define CM_MODE 3
#define CM_LAUNCH launch_sw16_w16_m3
#define CM_OCC sw16_occ_w16_m3
#include "sw16_inst.cuh"
