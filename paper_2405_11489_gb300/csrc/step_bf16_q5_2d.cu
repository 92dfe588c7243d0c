// Step kernel: storage __nv_bfloat16, arithmetic float, D1Q5-based lattice, 2d grids.
#define POND_S __nv_bfloat16
#define POND_R float
#define POND_Q1 5
#define POND_ONED false
#define POND_TAG bf16_q5_2d
#include "pond_step_inst.cuh"
