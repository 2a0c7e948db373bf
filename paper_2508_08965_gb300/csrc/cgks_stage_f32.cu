/* Stage launchers in FP32 (see cgks_stage.inc). */
#define CGKS_STAGE_T float
#include "cgks_stage.inc"
