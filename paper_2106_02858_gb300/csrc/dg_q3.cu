// Stage kernel instantiation for polynomial order 3.
#define CMCG_Q 3
#include "dg_stage.cuh"
