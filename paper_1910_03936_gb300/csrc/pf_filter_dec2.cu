#define PF_DEC 2
#include "pf_filter_inst.cuh"
