"""A whole Dirichlet problem through the C ABI: V_h, K_h assembly, data
projection, right-hand side (1/2 M_h + K_h) g, forward-substitution solve and
the relative L2(Sigma_h) error of the Neumann datum (Sec. 3.4, Sec. 6.1).

This module only allocates device buffers (torch) and calls the library in
order; all arithmetic happens in the CUDA kernels.
"""
import math

import torch

from . import capi


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class DirichletProblem:
    """Buffers and calls for one mesh / parameter set / list of sources.

    sources: numpy [nrhs, n_src, 5] of (y1, y2, y3, t0, weight).
    """

    def __init__(self, nodes, tris, alpha, T, n_steps, sources, quad_regular=3, quad_singular=4,
                 storage=capi.STB_STORE_F64, q_space=8, n_time=16, device="cuda", mesh=None,
                 precision=capi.STB_PREC_FP64):
        self.mesh = mesh if mesh is not None else capi.Mesh(nodes, tris)
        self.params = capi.stb_default_params(alpha, T, n_steps, quad_regular, quad_singular,
                                              precision=precision, storage=storage)
        self.sources = sources
        self.nrhs, self.n_src = sources.shape[0], sources.shape[1]
        self.q_space, self.n_time = q_space, n_time
        E, dev = self.mesh.n_tris, torch.device(device)
        self.E, self.n_steps, self.device = E, n_steps, dev
        dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
        self.V = torch.empty((n_steps, E, E), dtype=dt, device=dev)
        self.K = torch.empty((n_steps, E, E), dtype=dt, device=dev)
        vec = (self.nrhs, n_steps, E)
        self.g = torch.empty(vec, dtype=torch.float64, device=dev)
        self.f = torch.empty(vec, dtype=torch.float64, device=dev)
        self.w = torch.empty(vec, dtype=torch.float64, device=dev)
        self.err = torch.zeros(2, dtype=torch.float64, device=dev)
        m, p = self.mesh, self.params
        self.ws_assemble = _ws(capi.stb_assemble_workspace_size(m, p), dev)
        self.ws_project = _ws(capi.stb_project_workspace_size(m, self.nrhs, self.n_src, q_space, n_time), dev)
        self.ws_rhs = _ws(capi.stb_rhs_workspace_size(m, p, self.nrhs), dev)
        self.ws_solve = _ws(capi.stb_solve_workspace_size(m, p, self.nrhs), dev)
        self.ws_error = _ws(capi.stb_error_workspace_size(m, p, self.nrhs, self.n_src, q_space, n_time), dev)

    def assemble(self, stream=None):
        capi.stb_assemble(self.mesh, self.params, self.V, self.K, self.ws_assemble, stream)

    def project(self, stream=None):
        capi.stb_project_dirichlet(self.mesh, self.params, self.sources, self.g, self.ws_project,
                                   self.q_space, self.n_time, stream)

    def rhs(self, stream=None):
        capi.stb_dirichlet_rhs(self.mesh, self.params, self.K, self.g, self.nrhs, self.f,
                               self.ws_rhs, stream)

    def solve(self, stream=None):
        capi.stb_dirichlet_solve(self.mesh, self.params, self.V, self.f, self.nrhs, self.w,
                                 self.ws_solve, stream)

    def error(self, stream=None):
        capi.stb_neumann_error(self.mesh, self.params, self.sources, self.w, self.err, self.ws_error,
                               self.q_space, self.n_time, stream)

    def run(self, stream=None):
        """Every step of the path; returns the device tensor [err2, ref2]."""
        self.assemble(stream)
        self.project(stream)
        self.rhs(stream)
        self.solve(stream)
        self.error(stream)
        return self.err

    def relative_error(self):
        e = self.err.cpu()
        return math.sqrt(float(e[0]) / float(e[1]))
