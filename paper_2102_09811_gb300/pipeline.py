"""A whole Dirichlet problem through the C ABI: V_h, K_h assembly, data
projection, right-hand side (1/2 M_h + K_h) g, forward-substitution solve and
the relative L2(Sigma_h) error of the Neumann datum (Sec. 3.4, Sec. 6.1).

This module only allocates device buffers (torch) and calls the library in
order; all arithmetic happens in the CUDA kernels.
"""
import math

import numpy as np

import torch

from . import capi


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class DirichletProblem:
    """Buffers and calls for one mesh / parameter set / list of sources.

    sources: numpy [nrhs, n_src, 5] of (y1, y2, y3, t0, weight).
    data: "p0" projects the Dirichlet datum into piecewise constants in space
    (K_h with E x E blocks); "p1" into the continuous piecewise-linear space
    X_h^{1,0} (Sec. 3.2, Sec. 3.4: K_h with E x n_nodes blocks; the p0 x p1
    mass in the right-hand side).
    """

    def __init__(self, nodes, tris, alpha, T, n_steps, sources, quad_regular=3, quad_singular=4,
                 storage=capi.STB_STORE_F64, q_space=8, n_time=16, device="cuda", mesh=None,
                 precision=capi.STB_PREC_FP64, data="p0"):
        if data not in ("p0", "p1"):
            raise ValueError("data must be 'p0' or 'p1'")
        self.data = data
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
        N = self.mesh.n_nodes if data == "p1" else E
        self.K = torch.empty((n_steps, E, N), dtype=dt, device=dev)
        vec = (self.nrhs, n_steps, E)
        self.g = torch.empty((self.nrhs, n_steps, N), dtype=torch.float64, device=dev)
        self.f = torch.empty(vec, dtype=torch.float64, device=dev)
        self.w = torch.empty(vec, dtype=torch.float64, device=dev)
        self.err = torch.zeros(2, dtype=torch.float64, device=dev)
        m, p = self.mesh, self.params
        self.ws_assemble = _ws(capi.stb_assemble_workspace_size(m, p), dev)
        if data == "p1":
            # K1 in mixed precision where its FP32 storage allows, else FP64
            k1_prec = (capi.STB_PREC_MIXED if precision == capi.STB_PREC_MIXED and
                       storage == capi.STB_STORE_F32 else capi.STB_PREC_FP64)
            self.params_k1 = capi.stb_default_params(alpha, T, n_steps, quad_regular, quad_singular,
                                                     precision=k1_prec, storage=storage)
            self.ws_k1 = _ws(capi.stb_assemble_k1_workspace_size(m, self.params_k1), dev)
            self.ws_project = _ws(capi.stb_project_p1_workspace_size(m, p, self.nrhs, self.n_src,
                                                                     q_space, n_time), dev)
            self.ws_rhs = _ws(capi.stb_rhs_p1_workspace_size(m, p, self.nrhs), dev)
        else:
            self.ws_project = _ws(capi.stb_project_workspace_size(m, self.nrhs, self.n_src, q_space,
                                                                  n_time), dev)
            self.ws_rhs = _ws(capi.stb_rhs_workspace_size(m, p, self.nrhs), dev)
        self.ws_solve = _ws(capi.stb_solve_workspace_size(m, p, self.nrhs), dev)
        self.ws_error = _ws(capi.stb_error_workspace_size(m, p, self.nrhs, self.n_src, q_space, n_time), dev)

    def assemble(self, stream=None):
        if self.data == "p1":
            capi.stb_assemble(self.mesh, self.params, self.V, None, self.ws_assemble, stream)
            capi.stb_assemble_k1(self.mesh, self.params_k1, self.K, self.ws_k1, stream)
        else:
            capi.stb_assemble(self.mesh, self.params, self.V, self.K, self.ws_assemble, stream)

    def project(self, stream=None):
        fn = capi.stb_project_dirichlet_p1 if self.data == "p1" else capi.stb_project_dirichlet
        fn(self.mesh, self.params, self.sources, self.g, self.ws_project, self.q_space, self.n_time,
           stream)

    def rhs(self, stream=None):
        fn = capi.stb_dirichlet_rhs_p1 if self.data == "p1" else capi.stb_dirichlet_rhs
        fn(self.mesh, self.params, self.K, self.g, self.nrhs, self.f, self.ws_rhs, stream)

    def solve(self, stream=None):
        capi.stb_dirichlet_solve(self.mesh, self.params, self.V, self.f, self.nrhs, self.w,
                                 self.ws_solve, stream)

    def error(self, stream=None):
        capi.stb_neumann_error(self.mesh, self.params, self.sources, self.w, self.err, self.ws_error,
                               self.q_space, self.n_time, stream)

    def set_async(self, refinements):
        """From now on every call only enqueues device work: the solve runs
        `refinements` refinement steps (mixed precision; the count of an
        earlier synchronous solve) and leaves its convergence in the solve
        workspace's status word (STB_FLAG_NO_SYNC), the sources sit in
        page-locked memory so that their upload does not wait for the stream.
        Several problems can then run concurrently on their own streams."""
        self.params.flags = capi.STB_FLAG_NO_SYNC | capi.STB_FLAG_REFINE(max(1, refinements))
        if not hasattr(self.sources, "data_ptr"):
            self.sources = torch.tensor(self.sources, dtype=torch.float64).pin_memory()

    def solve_status(self):
        """(refinements, relative residual, status code) of the last solve."""
        r, res = capi.stb_solve_report(self.ws_solve)
        try:
            capi.stb_workspace_status(self.ws_solve)
            st = 0
        except capi.StbError as e:
            st = e.code
        return r, res, st

    def run(self, stream=None):
        """Every step of the path; returns the device tensor [err2, ref2]."""
        self.assemble(stream)
        self.project(stream)
        self.rhs(stream)
        self.solve(stream)
        self.error(stream)
        return self.err

    def representation(self, points, q_space=4, stream=None):
        """u_h = V~ w_h - W g_h at points [n_pts, 4] = (x1, x2, x3, t) inside
        the domain (eq. repr, Sec. 3.5), after run(); needs data="p1" (the
        double layer acts on the piecewise-linear Dirichlet data).  Returns
        a device tensor [nrhs, n_pts]."""
        if self.data != "p1":
            raise ValueError("the representation formula needs data='p1'")
        pts = torch.as_tensor(points, dtype=torch.float64).to(self.device).contiguous()
        n_pts = pts.shape[0]
        slp = torch.empty((self.nrhs, n_pts), dtype=torch.float64, device=self.device)
        dlp = torch.empty_like(slp)
        ws = _ws(capi.stb_potentials_workspace_size(self.mesh, self.params, self.nrhs, n_pts,
                                                    q_space), self.device)
        capi.stb_potentials(self.mesh, self.params, pts, self.w, self.g, self.nrhs, slp, dlp, ws,
                            q_space, stream)
        capi.stb_workspace_status(ws, stream)
        return slp - dlp

    def relative_error(self):
        e = self.err.cpu()
        return math.sqrt(float(e[0]) / float(e[1]))


class NeumannProblem:
    """The Neumann problem D_h u = (1/2 M_h^{T_x} - K_h^{T_x}) h (Sec. 3.3,
    Sec. 3.4) for exterior heat sources: Neumann data projected into
    X_h^{0,0}, the Dirichlet datum computed in X_h^{1,0}.  V (for D_h^1), K
    with piecewise-linear trial functions and D_h are assembled in the given
    precision where the library has it (D_h^2: FP64 arithmetic), stored in
    `storage`.
    """

    def __init__(self, nodes, tris, alpha, T, n_steps, sources, quad_regular=3, quad_singular=4,
                 storage=capi.STB_STORE_F64, q_space=8, n_time=16, device="cuda", mesh=None,
                 precision=capi.STB_PREC_FP64):
        self.mesh = mesh if mesh is not None else capi.Mesh(nodes, tris)
        mk = lambda prec: capi.stb_default_params(alpha, T, n_steps, quad_regular, quad_singular,
                                                  precision=prec, storage=storage)
        self.params = mk(precision)
        mixed_ok = precision == capi.STB_PREC_MIXED and storage == capi.STB_STORE_F32
        self.params_k1 = mk(capi.STB_PREC_MIXED if mixed_ok else capi.STB_PREC_FP64)
        self.params_d = mk(capi.STB_PREC_MIXED if mixed_ok else capi.STB_PREC_FP64)
        self.sources = sources
        self.nrhs, self.n_src = sources.shape[0], sources.shape[1]
        self.q_space, self.n_time = q_space, n_time
        E, N, dev = self.mesh.n_tris, self.mesh.n_nodes, torch.device(device)
        self.E, self.N, self.n_steps, self.device = E, N, n_steps, dev
        dt = torch.float64 if storage == capi.STB_STORE_F64 else torch.float32
        self.V = torch.empty((n_steps, E, E), dtype=dt, device=dev)
        self.K = torch.empty((n_steps, E, N), dtype=dt, device=dev)
        self.D = torch.empty((n_steps, N, N), dtype=dt, device=dev)
        self.hd = torch.empty((self.nrhs, n_steps, E), dtype=torch.float64, device=dev)
        self.f = torch.empty((self.nrhs, n_steps, N), dtype=torch.float64, device=dev)
        self.u = torch.empty((self.nrhs, n_steps, N), dtype=torch.float64, device=dev)
        self.err = torch.zeros(2, dtype=torch.float64, device=dev)
        m, p = self.mesh, self.params
        self.ws_v = _ws(capi.stb_assemble_workspace_size(m, p), dev)
        self.ws_k1 = _ws(capi.stb_assemble_k1_workspace_size(m, self.params_k1), dev)
        self.ws_d = _ws(capi.stb_assemble_d_workspace_size(m, self.params_d), dev)
        self.ws_project = _ws(capi.stb_project_workspace_size(m, self.nrhs, self.n_src, q_space,
                                                              n_time), dev)
        self.ws_rhs = _ws(capi.stb_neumann_rhs_workspace_size(m, p, self.nrhs), dev)
        self.ws_solve = _ws(capi.stb_neumann_solve_workspace_size(m, p, self.nrhs), dev)
        self.ws_error = _ws(capi.stb_error_workspace_size(m, p, self.nrhs, self.n_src, q_space,
                                                          n_time), dev)

    def assemble(self, stream=None):
        capi.stb_assemble(self.mesh, self.params, self.V, None, self.ws_v, stream)
        capi.stb_assemble_k1(self.mesh, self.params_k1, self.K, self.ws_k1, stream)
        capi.stb_assemble_d(self.mesh, self.params_d, self.V, self.D, self.ws_d, stream)

    def project(self, stream=None):
        capi.stb_project_neumann(self.mesh, self.params, self.sources, self.hd, self.ws_project,
                                 self.q_space, self.n_time, stream)

    def rhs(self, stream=None):
        capi.stb_neumann_rhs(self.mesh, self.params, self.K, self.hd, self.nrhs, self.f,
                             self.ws_rhs, stream)

    def solve(self, stream=None):
        capi.stb_neumann_solve(self.mesh, self.params, self.D, self.f, self.nrhs, self.u,
                               self.ws_solve, stream)

    def error(self, stream=None):
        capi.stb_dirichlet_error_p1(self.mesh, self.params, self.sources, self.u, self.err,
                                    self.ws_error, self.q_space, self.n_time, stream)

    def run(self, stream=None):
        self.assemble(stream)
        self.project(stream)
        self.rhs(stream)
        self.solve(stream)
        self.error(stream)
        return self.err

    def relative_error(self):
        e = self.err.cpu()
        return math.sqrt(float(e[0]) / float(e[1]))

    def representation(self, points, q_space=4, stream=None):
        """u_h = V~ h_h - W u_h at points [n_pts, 4] inside the domain."""
        pts = torch.as_tensor(points, dtype=torch.float64).to(self.device).contiguous()
        n_pts = pts.shape[0]
        slp = torch.empty((self.nrhs, n_pts), dtype=torch.float64, device=self.device)
        dlp = torch.empty_like(slp)
        ws = _ws(capi.stb_potentials_workspace_size(self.mesh, self.params, self.nrhs, n_pts,
                                                    q_space), self.device)
        capi.stb_potentials(self.mesh, self.params, pts, self.hd, self.u, self.nrhs, slp, dlp, ws,
                            q_space, stream)
        capi.stb_workspace_status(ws, stream)
        return slp - dlp


class NonUniformDirichletProblem:
    """The Dirichlet problem on a non-uniform time grid `times` (Sec. 7):
    block lower-triangular V, K with packed blocks (FP64; precision
    STB_PREC_MIXED evaluates the quadrature points in FP32), data projection over the steps,
    right-hand side, forward substitution with a factorisation per diagonal
    block, and the L2(Sigma_h) error."""

    def __init__(self, nodes, tris, alpha, times, sources, quad_regular=3, quad_singular=4,
                 q_space=8, n_time=16, device="cuda", mesh=None, precision=capi.STB_PREC_FP64):
        self.mesh = mesh if mesh is not None else capi.Mesh(nodes, tris)
        self.times = np.ascontiguousarray(times, dtype=np.float64)
        n = len(self.times) - 1
        self.params = capi.stb_default_params(alpha, float(self.times[-1]), n, quad_regular,
                                              quad_singular, precision=precision)
        self.sources = sources
        self.nrhs, self.n_src = sources.shape[0], sources.shape[1]
        self.q_space, self.n_time = q_space, n_time
        E, dev = self.mesh.n_tris, torch.device(device)
        self.E, self.n_steps, self.device = E, n, dev
        nblk = n * (n + 1) // 2
        self.V = torch.empty((nblk, E, E), dtype=torch.float64, device=dev)
        self.K = torch.empty((nblk, E, E), dtype=torch.float64, device=dev)
        vec = (self.nrhs, n, E)
        self.g = torch.empty(vec, dtype=torch.float64, device=dev)
        self.f = torch.empty(vec, dtype=torch.float64, device=dev)
        self.w = torch.empty(vec, dtype=torch.float64, device=dev)
        self.err = torch.zeros(2, dtype=torch.float64, device=dev)
        m, p = self.mesh, self.params
        self.ws_assemble = _ws(capi.stb_assemble_nu_workspace_size(m, p, self.times), dev)
        self.ws_data = _ws(capi.stb_project_nu_workspace_size(m, p, self.nrhs, self.n_src, q_space,
                                                              n_time), dev)
        self.ws_rhs = _ws(capi.stb_dirichlet_rhs_nu_workspace_size(m, p), dev)
        self.ws_solve = _ws(capi.stb_solve_nu_workspace_size(E, n, self.nrhs), dev)

    def run(self, stream=None):
        m, p, t = self.mesh, self.params, self.times
        capi.stb_assemble_nu(m, p, t, self.V, self.K, self.ws_assemble, stream)
        capi.stb_project_dirichlet_nu(m, p, t, self.sources, self.g, self.ws_data, self.q_space,
                                      self.n_time, stream)
        capi.stb_dirichlet_rhs_nu(m, p, t, self.K, self.g, self.nrhs, self.f, self.ws_rhs, stream)
        capi.stb_solve_nu(self.V, self.E, self.n_steps, self.nrhs, self.f, self.w, self.ws_solve,
                          stream)
        capi.stb_neumann_error_nu(m, p, t, self.sources, self.w, self.err, self.ws_data,
                                  self.q_space, self.n_time, stream)
        return self.err

    def relative_error(self):
        e = self.err.cpu()
        return math.sqrt(float(e[0]) / float(e[1]))


class BatchPipeline:
    """Many independent Dirichlet problems, mixed precision, FP32 storage.

    problems: list of dicts with nodes, tris, alpha, T, n_steps, sources.
    The problems are grouped into waves whose V and K fit `wave_bytes` (one
    arena of that size, shared by the waves).  Per wave, stb_batch_prepare
    uploads the tables once; everything after it -- the batched assembly
    launches, and per problem the projection, right-hand side, solve (with
    the refinement count of a first, synchronous pass) and error -- is captured
    into one CUDA graph on the first run and replayed on later runs.  The
    captured calls carry STB_FLAG_NO_SYNC; sources are kept in page-locked
    host memory.
    """

    def __init__(self, problems, wave_bytes=48e9, device="cuda", tile=0, tune=True,
                 q_space=8, n_time=16):
        dev = torch.device(device)
        self.device, self.q_space, self.n_time, self.tile, self.tune = dev, q_space, n_time, tile, tune
        self.items = []
        for p in problems:
            mesh = capi.Mesh(p["nodes"], p["tris"])
            prm = capi.stb_default_params(p["alpha"], p["T"], p["n_steps"],
                                          precision=capi.STB_PREC_MIXED, storage=capi.STB_STORE_F32)
            src = torch.tensor(p["sources"], dtype=torch.float64).pin_memory()
            nrhs, n_src = src.shape[0], src.shape[1]
            E, n = mesh.n_tris, p["n_steps"]
            vec = (nrhs, n, E)
            it = dict(mesh=mesh, params=prm, sources=src, E=E, n_steps=n, nrhs=nrhs,
                      g=torch.zeros(vec, dtype=torch.float64, device=dev),
                      f=torch.zeros(vec, dtype=torch.float64, device=dev),
                      w=torch.zeros(vec, dtype=torch.float64, device=dev),
                      err=torch.zeros(2, dtype=torch.float64, device=dev),
                      ws_solve=_ws(capi.stb_solve_workspace_size(mesh, prm, nrhs), dev),
                      vk_bytes=8 * E * E * n)
            it["ws_project"] = capi.stb_project_workspace_size(mesh, nrhs, n_src, q_space, n_time)
            it["ws_rhs"] = capi.stb_rhs_workspace_size(mesh, prm, nrhs)
            it["ws_error"] = capi.stb_error_workspace_size(mesh, prm, nrhs, n_src, q_space, n_time)
            self.items.append(it)
        order = sorted(range(len(self.items)), key=lambda i: -self.items[i]["vk_bytes"])
        self.waves, cur, size = [], [], 0
        for i in order:
            b = self.items[i]["vk_bytes"]
            if b > wave_bytes:
                raise ValueError("problem %d needs %d bytes of blocks, more than wave_bytes" % (i, b))
            if cur and size + b > wave_bytes:
                self.waves.append(cur)
                cur, size = [], 0
            cur.append(i)
            size += b
        if cur:
            self.waves.append(cur)
        arena = max(sum(self.items[i]["vk_bytes"] for i in w) for w in self.waves)
        self.arena = torch.empty(arena // 4, dtype=torch.float32, device=dev)
        shared = max(max(it["ws_project"], it["ws_rhs"], it["ws_error"]) for it in self.items)
        self.ws_shared = _ws(shared, dev)
        self.graphs = [None] * len(self.waves)
        self.graph_launches = [0] * len(self.waves)  # library kernels per replay
        self.wave_state = [None] * len(self.waves)

    def _wave_buffers(self, w):
        """V, K views of the arena for the problems of wave w."""
        V, K, off = [], [], 0
        for i in self.waves[w]:
            it = self.items[i]
            n = it["n_steps"] * it["E"] * it["E"]
            V.append(self.arena[off:off + n].view(it["n_steps"], it["E"], it["E"]))
            K.append(self.arena[off + n:off + 2 * n].view(it["n_steps"], it["E"], it["E"]))
            off += 2 * n
        return V, K

    def _enqueue(self, w, stream):
        """The capturable part of wave w (after stb_batch_prepare)."""
        meshes, params, V, K, tile, ws = self.wave_state[w]
        capi.stb_batch_launch(meshes, params, V, K, tile, ws, stream)
        for k, i in enumerate(self.waves[w]):
            it = self.items[i]
            m, p = it["mesh"], it["params"]
            capi.stb_project_dirichlet(m, p, it["sources"], it["g"], self.ws_shared, self.q_space,
                                       self.n_time, stream)
            capi.stb_dirichlet_rhs(m, p, K[k], it["g"], it["nrhs"], it["f"], self.ws_shared, stream)
            capi.stb_dirichlet_solve(m, p, V[k], it["f"], it["nrhs"], it["w"], it["ws_solve"],
                                     stream)
            capi.stb_neumann_error(m, p, it["sources"], it["w"], it["err"], self.ws_shared,
                                   self.q_space, self.n_time, stream)

    def _build(self, w, stream):
        meshes = [self.items[i]["mesh"] for i in self.waves[w]]
        params = [self.items[i]["params"] for i in self.waves[w]]
        V, K = self._wave_buffers(w)
        ws = _ws(capi.stb_batch_workspace_size(meshes, params, V, K), self.device)
        tile = self.tile
        if tile == 0 and self.tune:
            tile = capi.stb_batch_tune(meshes, params, V, K, ws, stream)
        capi.stb_batch_prepare(meshes, params, V, K, tile, ws, stream)
        self.wave_state[w] = (meshes, params, V, K, tile, ws)
        # one uncaptured pass with synchronous solves: builds the page-locked
        # rule tables and gives each problem's refinement count, which the
        # captured solves then run without host synchronisation
        for p in params:
            p.flags = 0
        self._enqueue(w, stream)
        torch.cuda.synchronize()
        for i, p in zip(self.waves[w], params):
            r, _ = capi.stb_solve_report(self.items[i]["ws_solve"])
            p.flags = capi.STB_FLAG_NO_SYNC | capi.STB_FLAG_REFINE(max(1, r))
        g = torch.cuda.CUDAGraph()
        n0 = capi.stb_launch_count()
        with torch.cuda.graph(g):
            self._enqueue(w, torch.cuda.current_stream())
        self.graph_launches[w] = capi.stb_launch_count() - n0
        self.graphs[w] = g

    def run(self, stream=None):
        """All waves: replays each wave's graph (built on the first call)."""
        s = stream if stream is not None else torch.cuda.current_stream()
        for w in range(len(self.waves)):
            if self.graphs[w] is None:
                self._build(w, s)
            self.graphs[w].replay()

    def relative_errors(self):
        return [math.sqrt(float(e[0]) / float(e[1])) for e in (it["err"].cpu() for it in self.items)]

    def reports(self):
        """(refinements, relative residual, status) of every problem's solve."""
        out = []
        for it in self.items:
            r, res = capi.stb_solve_report(it["ws_solve"])
            try:
                capi.stb_workspace_status(it["ws_solve"])
                st = 0
            except capi.StbError as e:
                st = e.code
            out.append((r, res, st))
        return out
