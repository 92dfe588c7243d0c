// Step kernel: storage double, arithmetic double, D1Q5-based lattice, 2d grids.
#define POND_S double
#define POND_R double
#define POND_Q1 5
#define POND_ONED false
#define POND_TAG f64_q5_2d
#include "pond_step_inst.cuh"
