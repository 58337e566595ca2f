// Double-float hexahedral operator kernels of degree p = 4 (R, J v, J^T w, block columns).
#include "enp_op_dispatch.cuh"
ENP_DF_DEGREE(4)
