// Launch shape 3 of the box-sum sweep (shapes listed in sweep_box.cuh).
#include "sweep_box.cuh"

TNLM_BOX_VARIANT_TU(3)
