// qc_dd_stream_delay.cu -- streaming kernels of chains with directions: solved delay terms (parameter sums).
#include "qc_dd_stream_inst.cuh"

DDSLaunch dds_launcher_delay(int ok, bool oleft) { return qc_dds::pick<qc::KIND_DIAG, true, 0>(ok, oleft); }
