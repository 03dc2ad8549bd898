"""Writes sinpi_poly.h: coefficients of an odd polynomial z*p(z^2) approximating
sin(pi z / 2) on z in [-1, 1], fitted here by least squares on Chebyshev nodes in
float64 (no library coefficients are used).  Run: python gen_sinpi.py > sinpi_poly.h"""
import numpy as np

DEG = 6  # terms z, z^3, ..., z^11
n = 4001
z = np.cos(np.pi * (np.arange(n) + 0.5) / n)  # Chebyshev nodes on [-1, 1]
z = z[z > 0]
f = np.sin(np.pi * z / 2)
A = np.stack([z ** (2 * k + 1) for k in range(DEG)], axis=1)
c, *_ = np.linalg.lstsq(A, f, rcond=None)
c32 = c.astype(np.float32)
zz = np.linspace(-1, 1, 200001).astype(np.float32)
z2 = zz * zz
acc = np.float32(c32[-1])
for k in range(DEG - 2, -1, -1):
    acc = (acc * z2 + c32[k]).astype(np.float32)
err = np.max(np.abs(acc.astype(np.float64) * zz - np.sin(np.pi * zz.astype(np.float64) / 2)))
print("// Generated by gen_sinpi.py: sin(pi z / 2) ~= z * (c0 + z^2 (c1 + z^2 (c2 + ...))), |z| <= 1")
print(f"// max abs error in float32 evaluation: {err:.2e}")
print("#pragma once")
for k, v in enumerate(c32):
    print(f"#define RECON_SINPI_C{k} {float(v)!r}f")
