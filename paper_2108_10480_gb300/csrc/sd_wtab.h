// Layout of the nested-Horner tables of the triangle weight (App. C.3),
// shared by the host code that computes them and the kernels that read them.
#pragma once

// classes (v, e): vertex valence v = 1..SD_WT_VMAX, edge valence e = 1..SD_WT_EMAX
#define SD_WT_VMAX 16
#define SD_WT_EMAX 4
// floats per (class, orientation): 36 (w~) + 28 (dw~/dphi1) + 28 (dw~/dphi2)
#define SD_WT_FLOATS 92
#define SD_WT_CLASSES (SD_WT_VMAX * SD_WT_EMAX * 3 * SD_WT_FLOATS)
// after the class tables, the same for the three parts of the blend
// (base = P_B, dv = P_V - P_B, de = P_E: w~ = base + dv / v + de / e), used
// for classes outside the table
#define SD_WT_TOTAL (SD_WT_CLASSES + 3 * 3 * SD_WT_FLOATS)

// out[SD_WT_TOTAL]; class (v, e), orientation o at ((v-1) * SD_WT_EMAX + (e-1)) * 3 + o
extern "C" int sd_weight_horner_tables(float* out);
// out[3 * 3 * SD_WT_FLOATS]: base, dv, de, each 3 orientations
int sd_weight_horner_basis(float* out);
