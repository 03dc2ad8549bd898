// Generated by gen_sinpi.py: sin(pi z / 2) ~= z * (c0 + z^2 (c1 + z^2 (c2 + ...))), |z| <= 1
// max abs error in float32 evaluation: 1.73e-07
#pragma once
#define RECON_SINPI_C0 1.5707963705062866f
#define RECON_SINPI_C1 -0.6459640860557556f
#define RECON_SINPI_C2 0.07969258725643158f
#define RECON_SINPI_C3 -0.00468162028118968f
#define RECON_SINPI_C4 0.00016021713963709772f
#define RECON_SINPI_C5 -3.418172809688258e-06f
