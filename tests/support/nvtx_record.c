/* NVTX injection library for the tests: records every range pushed with nvtxRangePushA (and every pop)
 * into the file named by LABS_NVTX_LOG.  Loaded by NVTX through NVTX_INJECTION64_PATH. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE* g_log;

static int record_push(const char* msg) {
  if (g_log) {
    fprintf(g_log, "push %s\n", msg ? msg : "");
    fflush(g_log);
  }
  return 0;
}

static int record_pop(void) {
  if (g_log) {
    fputs("pop\n", g_log);
    fflush(g_log);
  }
  return 0;
}

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  const char* path = getenv("LABS_NVTX_LOG");
  if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
  if (size > NVTX_CBID_CORE_RangePushA) *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
  if (size > NVTX_CBID_CORE_RangePop) *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
  if (path) g_log = fopen(path, "w");
  return 1;
}
