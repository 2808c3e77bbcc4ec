// int16x2 kernel instantiations: CTAs of 8 warps, launch mode 1 (SwMode).
#define CM_W 8
#define CM_MODE 1
#define CM_LAUNCH launch_sw16_w8_m1
#define CM_OCC sw16_occ_w8_m1
#include "sw16_inst.cuh"
