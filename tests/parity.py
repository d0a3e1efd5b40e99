"""Shared helpers of the GPU parity tests: run a workload through libfe and the
oracle on the same seeded inputs and measure the relative errors."""
import numpy as np

import oracle
from paper_2107_04121_gb300 import fe

TOL = {"f64": 1e-12, "f32": 1e-5, "tf32x3": 1e-5, "bf16x3": 1e-5}


def rel_matrix_error(K, Kref):
    """max over elements of ||K_e - K_e^ref||_F / ||K_e^ref||_F."""
    K = np.asarray(K, dtype=np.float64)
    num = np.sqrt(((K - Kref) ** 2).sum((1, 2)))
    den = np.sqrt((Kref ** 2).sum((1, 2)))
    return float((num / den).max()) if len(den) else 0.0


def rel_vector_error(r, rref):
    """||r - r_ref||_2 / ||r_ref||_2 over the whole array."""
    r = np.asarray(r, dtype=np.float64).ravel()
    rref = np.asarray(rref).ravel()
    return float(np.linalg.norm(r - rref) / np.linalg.norm(rref))


class Problem:
    """A mesh with its GPU geometry and its oracle geometry."""

    def __init__(self, ctx, mesh, p, nq, device="cuda"):
        import torch
        self.ctx, self.mesh, self.p, self.nq = ctx, mesh, p, nq
        self.coords_d = torch.from_numpy(mesh.coords).to(device)
        self.conn_d = torch.from_numpy(mesh.conn).to(device)
        self.m = fe.Mesh(self.coords_d, self.conn_d)
        self.geom = fe.hex_geometry(ctx, self.m, p, nq)
        self.ref = oracle.RefElement(p, nq)
        self._ogeo = None

    def oracle_geometry(self, elems=None):
        conn = self.mesh.conn if elems is None else self.mesh.conn[elems]
        return oracle.geometry(self.mesh.coords, conn, self.ref)
