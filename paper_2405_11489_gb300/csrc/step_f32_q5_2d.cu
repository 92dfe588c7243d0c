// Step kernel: storage float, arithmetic float, D1Q5-based lattice, 2d grids.
#define POND_S float
#define POND_R float
#define POND_Q1 5
#define POND_ONED false
#define POND_TAG f32_q5_2d
#include "pond_step_inst.cuh"
