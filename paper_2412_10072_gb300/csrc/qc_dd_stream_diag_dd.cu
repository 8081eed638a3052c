// qc_dd_stream_diag_dd.cu -- streaming kernels of chains with directions: direction-dependent diagonal solved terms, two directions per CTA.
#include "qc_dd_stream_inst.cuh"

DDSLaunch dds_launcher_diag_dd(int ok, bool oleft) { return qc_dds::pick<qc::KIND_DIAG, false, 2>(ok, oleft); }
