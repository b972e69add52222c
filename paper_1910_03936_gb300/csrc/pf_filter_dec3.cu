#define PF_DEC 3
#include "pf_filter_inst.cuh"
