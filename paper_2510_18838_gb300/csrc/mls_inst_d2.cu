// Kernel instantiations of the 2D MLS transfer.
#include "mls_dispatch.cuh"

PCMS_DEFINE_MLS_DISPATCH(2)
