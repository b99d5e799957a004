#include "handle.h"
int hsw_factor(hsweep_s* h) { (void)h; return HSWEEP_ERR_ARG; }
void hsw_setup_free(hsweep_s* h) { (void)h; }
