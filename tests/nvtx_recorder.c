/* Test-only NVTX handler: records the core range calls of the library under test as text lines,
 * so a test can check the names and the nesting of the library's NVTX ranges without a profiler.
 * Loaded by NVTX itself through NVTX_INJECTION64_PATH (the documented injection entry point
 * InitializeInjectionNvtx2 fills the core function table), read back by the test through ctypes
 * with nvtx_recorder_log().  Lines: "push <name>", "pop", "start <id> <name>", "end <id>". */
#include <nvtx3/nvToolsExt.h>
#include <pthread.h>
#include <stdio.h>
#include <string.h>

static char g_log[1 << 20];
static size_t g_len = 0;
static uint64_t g_next_id = 1;
static pthread_mutex_t g_mu = PTHREAD_MUTEX_INITIALIZER;

static void append(const char* line) {
  pthread_mutex_lock(&g_mu);
  size_t n = strlen(line);
  if (g_len + n + 2 < sizeof(g_log)) {
    memcpy(g_log + g_len, line, n);
    g_len += n;
    g_log[g_len++] = '\n';
    g_log[g_len] = 0;
  }
  pthread_mutex_unlock(&g_mu);
}

static int NVTX_API rec_push(const char* name) {
  char line[512];
  snprintf(line, sizeof(line), "push %s", name ? name : "");
  append(line);
  return 0;
}

static int NVTX_API rec_pop(void) {
  append("pop");
  return 0;
}

static nvtxRangeId_t NVTX_API rec_start(const char* name) {
  char line[512];
  pthread_mutex_lock(&g_mu);
  const uint64_t id = g_next_id++;
  pthread_mutex_unlock(&g_mu);
  snprintf(line, sizeof(line), "start %llu %s", (unsigned long long)id, name ? name : "");
  append(line);
  return id;
}

static void NVTX_API rec_end(nvtxRangeId_t id) {
  char line[64];
  snprintf(line, sizeof(line), "end %llu", (unsigned long long)id);
  append(line);
}

const char* nvtx_recorder_log(void) { return g_log; }

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_export_table) {
  const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_export_table(NVTX_ETID_CALLBACKS);
  if (!cb || !cb->GetModuleFunctionTable) return 0;
  NvtxFunctionTable table = 0;
  unsigned int size = 0;
  if (!cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
  if (size <= NVTX_CBID_CORE_RangePop) return 0;
  *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)rec_push;
  *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)rec_pop;
  *table[NVTX_CBID_CORE_RangeStartA] = (NvtxFunctionPointer)rec_start;
  *table[NVTX_CBID_CORE_RangeEnd] = (NvtxFunctionPointer)rec_end;
  return 1;
}
