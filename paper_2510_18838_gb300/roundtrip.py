"""Vertex <-> centroid round trips on a triangle mesh: the accuracy (Eq. 2) and conservation
(Eq. 3) study of Sec. 3.2.1, run through the library.

One iteration takes a nodal field vertices -> centroids, then centroids -> vertices,
with two cached MLS operators (pcms_create_map), applied without allocation
(pcms_apply_map_noalloc) so that an iteration can be captured once in a CUDA graph and
replayed. The centroids (pcms_mesh_centroids) and the integral of the piecewise-linear
interpolant that Eq. 3 needs (pcms_mesh_integrate) are library kernels too. Per
iteration:
  accuracy     ||f - f*|| / ||f*|| over the vertices (L2, and L-infinity),
  conservation |I(f) - I(f*)| / |I(f*)|, I = integral of the P1 interpolant,
with f* the field before the first transfer. The paper leaves the norm of Eq. 2 open; L2
over the vertices is the reading used. The operators are FP64 (the study is about the
method's error, not rounding).
"""
from __future__ import annotations

import numpy as np
import torch

from . import pcms


def sincos_plus_two(xy) -> np.ndarray:
    """The study's smooth test field f(x, y) = sin(x) cos(y) + 2 (Sec. 3.2.1)."""
    xy = np.asarray(xy, np.float64)
    return np.sin(xy[0]) * np.cos(xy[1]) + 2.0


class RoundTrip:
    """Operators and buffers of the round trip on one mesh (device resident)."""

    def __init__(self, xy, tri, degree, radius, weight="c4", min_neighbors=0, stream=None):
        dev = torch.device("cuda", torch.cuda.current_device())
        self.xy = torch.as_tensor(np.ascontiguousarray(xy, np.float64)).to(dev) \
            if not isinstance(xy, torch.Tensor) else xy.to(dev, torch.float64).contiguous()
        self.tri = torch.as_tensor(np.ascontiguousarray(tri, np.int32)).to(dev) \
            if not isinstance(tri, torch.Tensor) else tri.to(dev, torch.int32).contiguous()
        self.stream = stream
        self.mesh = pcms.Mesh(self.xy, self.tri, stream=stream)
        self.centroids = self.mesh.centroids(stream=stream).contiguous()
        self.v2c = pcms.create_map(self.xy, self.centroids, degree, radius, weight=weight,
                                   min_neighbors=min_neighbors, stream=stream)
        self.c2v = pcms.create_map(self.centroids, self.xy, degree, radius, weight=weight,
                                   min_neighbors=min_neighbors, stream=stream)
        self.fv = torch.zeros(self.xy.shape[1], dtype=torch.float64, device=dev)
        self.fc = torch.zeros(self.tri.shape[1], dtype=torch.float64, device=dev)
        self.graph = None

    def load(self, f) -> None:
        """Set the vertex field (float64 [n_vertices])."""
        self.fv.copy_(torch.as_tensor(np.asarray(f, np.float64)) if not isinstance(f, torch.Tensor)
                      else f.to(torch.float64))

    def iterate(self, n: int = 1) -> None:
        """n iterations, vertices -> centroids -> vertices, launched one by one."""
        for _ in range(n):
            self.v2c.apply_noalloc(self.fv, self.fc, stream=self.stream)
            self.c2v.apply_noalloc(self.fc, self.fv, stream=self.stream)

    def capture(self) -> None:
        """Capture one iteration in a CUDA graph (its launches read and write the
        operator's own buffers, so replays chain)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        saved = self.fv.clone()
        with torch.cuda.stream(s):
            self.v2c.apply_noalloc(self.fv, self.fc, stream=s)   # first use outside capture
            self.c2v.apply_noalloc(self.fc, self.fv, stream=s)
        torch.cuda.current_stream().wait_stream(s)
        self.fv.copy_(saved)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
            self.v2c.apply_noalloc(self.fv, self.fc, stream=s)
            self.c2v.apply_noalloc(self.fc, self.fv, stream=s)
        self.graph = g

    def replay(self, n: int = 1) -> None:
        if self.graph is None:
            self.capture()
        for _ in range(n):
            self.graph.replay()

    def integral(self, f=None) -> float:
        return self.mesh.integrate(self.fv if f is None else f, stream=self.stream)

    def destroy(self):
        for m in (self.v2c, self.c2v):
            m.destroy()
        self.mesh.destroy()


def run(xy, tri, f_star, degree, radius, weight="c4", iterations=10, min_neighbors=0,
        graph=True) -> dict:
    """The study: per-iteration accuracy (L2, L-infinity) and conservation errors, and the
    final vertex field. Mirrors the oracle's round_trip output."""
    rt = RoundTrip(xy, tri, degree, radius, weight, min_neighbors)
    f_star = np.asarray(f_star, np.float64)
    rt.load(f_star)
    dev_star = rt.fv.clone()
    i_star = rt.integral(dev_star)
    if graph:
        rt.capture()
    n2, ninf = np.linalg.norm(f_star), np.abs(f_star).max()
    acc2 = np.empty(iterations)
    accinf = np.empty(iterations)
    cons = np.empty(iterations)
    for k in range(iterations):
        if graph:
            rt.replay(1)
        else:
            rt.iterate(1)
        f = rt.fv.cpu().numpy()
        acc2[k] = np.linalg.norm(f - f_star) / n2
        accinf[k] = np.abs(f - f_star).max() / ninf
        cons[k] = abs(rt.integral() - i_star) / abs(i_star)
    out = dict(accuracy_l2=acc2, accuracy_linf=accinf, conservation=cons,
               field=rt.fv.cpu().numpy(), integral_star=i_star)
    rt.destroy()
    return out
