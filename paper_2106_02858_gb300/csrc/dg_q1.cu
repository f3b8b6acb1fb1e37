// Stage kernel instantiation for polynomial order 1.
#define CMCG_Q 1
#include "dg_stage.cuh"
