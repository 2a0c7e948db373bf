/* Stage launchers in FP64 (see cgks_stage.inc). */
#define CGKS_STAGE_T double
#include "cgks_stage.inc"
