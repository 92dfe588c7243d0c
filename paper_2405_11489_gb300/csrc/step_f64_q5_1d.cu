// Step kernel: storage double, arithmetic double, D1Q5-based lattice, 1d grids.
#define POND_S double
#define POND_R double
#define POND_Q1 5
#define POND_ONED true
#define POND_TAG f64_q5_1d
#include "pond_step_inst.cuh"
