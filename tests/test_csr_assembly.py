"""The library's CSR assembly of a stencil matrix (stencil_csr, from the
coefficients gadi_create uses) equals the matrix assembled here from the
oracle's own coefficients, entry for entry (host only, no GPU)."""
import numpy as np
import pytest

import oracle as O
import paper_2512_21164_gb300 as G
from workloads import conv_diff_2d, conv_diff_3d


def oracle_csr(p):
    """CSR of A by the oracle's coefficients, assembled point by point."""
    co = O.Oracle(p).coeffs(0)  # centre, W, E, S, N, B, T, e
    nx, ny = p.nx, p.ny
    nz = p.nz if p.kind == O.K_3D7 else 1
    rp, cl, vl = [0], [], []
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                i = (iz * ny + iy) * nx + ix
                row = {i: co[0]}
                if ix > 0: row[i - 1] = co[1]
                if ix < nx - 1: row[i + 1] = co[2]
                if iy > 0: row[i - nx] = co[3]
                if iy < ny - 1: row[i + nx] = co[4]
                if nz > 1 and iz > 0: row[i - nx * ny] = co[5]
                if nz > 1 and iz < nz - 1: row[i + nx * ny] = co[6]
                for j in sorted(row):
                    cl.append(j)
                    vl.append(row[j])
                rp.append(len(cl))
    return np.asarray(rp, np.int32), np.asarray(cl, np.int32), np.asarray(vl, np.float64)


@pytest.mark.parametrize("mk", [lambda: conv_diff_2d(13, 5, ny=9), lambda: conv_diff_3d(5, 6),
                                lambda: conv_diff_2d(1, 7, ny=4)])
def test_stencil_csr_matches_oracle_assembly(mk):
    from paper_2512_21164_gb300 import build
    build.build()
    p, _ = mk()
    got = G.stencil_csr(p)
    want = oracle_csr(p)
    for a, b in zip(got, want):
        assert a.dtype == b.dtype and np.array_equal(a, b)
