/* NVTX injection library used by tests/test_trace_host.py (test
 * infrastructure).  Loaded through NVTX_INJECTION64_PATH, it takes over the
 * range push/pop callbacks and appends "push <name>" / "pop" lines to the
 * file named by CT_NVTX_LOG. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE *log_file;
static int depth;

static int NVTX_API probe_push(const char *message) {
    if (log_file) {
        fprintf(log_file, "push %s\n", message ? message : "");
        fflush(log_file);
    }
    return depth++;
}

static int NVTX_API probe_pop(void) {
    if (log_file) {
        fputs("pop\n", log_file);
        fflush(log_file);
    }
    return --depth;
}

int NVTX_API InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks *cb =
        (const NvtxExportTableCallbacks *)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size)) return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)probe_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)probe_pop;
    const char *path = getenv("CT_NVTX_LOG");
    log_file = path ? fopen(path, "w") : NULL;
    return 1;
}
