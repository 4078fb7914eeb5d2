// Process tables emitted by the process compiler (generated include).
#include "mg_internal.h"
#include "mg_tables.inc"

extern "C" const mg_proc_table *mg_tables(int *count) {
    if (count) *count = MG_NPROC_TABLES;
    return MG_PROC_TABLES;
}
