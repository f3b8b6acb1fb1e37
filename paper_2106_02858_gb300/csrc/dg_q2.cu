// Stage kernel instantiation for polynomial order 2.
#define CMCG_Q 2
#include "dg_stage.cuh"
