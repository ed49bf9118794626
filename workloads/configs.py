"""The five synthetic workloads (sizes, maps, media, runs).

They stand in for the paper's LOH1 and Zugspitze experiments (Section 7),
whose reference seismograms and topography data are not available: same
regime (layered / topographic / h of order 100 m, point moment-tensor
sources, surface stations), synthetic seeded data.

Faces are numbered (q=0, q=1, r=0, r=1, s=0, s=1).  The top surface is s=1.
A boundary entry is ("free",) for the free-surface penalty or
("char", gamma) for the characteristic penalty with parameter gamma.
"""
from dataclasses import dataclass, field

ABSORB = ("char", 0.0)
FREE = ("free",)


@dataclass(frozen=True)
class WorkloadConfig:
    name: str
    nodes: tuple            # (nq, nr, ns)
    extent: tuple           # (Lx, Ly, Lz) in metres
    geometry: str           # identity | gaussian_hill | sinusoids
    order: int              # interior order of the upwind pair: 2, 4 or 6
    precisions: tuple       # solver precisions exercised (bits)
    medium: str             # homogeneous | layered3 | gradient_vonkarman
    steps: int
    cfl: float = 0.5
    n_receivers: int = 0
    initial: str = "zero"   # zero | gaussian_pulse | smooth_random
    source: str = "none"    # none | moment_tensor
    seed: int = 0
    bc: tuple = (ABSORB, ABSORB, ABSORB, ABSORB, ABSORB, FREE)
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return self.nodes[0] * self.nodes[1] * self.nodes[2]


CONFIGS = [
    WorkloadConfig(
        name="cube33_o4_fp64", nodes=(33, 33, 33), extent=(1000.0, 1000.0, 1000.0),
        geometry="identity", order=4, precisions=(64,), medium="homogeneous",
        steps=100, n_receivers=4, initial="gaussian_pulse",
        extra=dict(pulse_width=50.0)),
    WorkloadConfig(
        name="hill129_o6", nodes=(129, 129, 97), extent=(20000.0, 20000.0, 15000.0),
        geometry="gaussian_hill", order=6, precisions=(64, 32), medium="layered3",
        steps=2000, n_receivers=16, source="moment_tensor",
        extra=dict(hill_amp=1500.0, hill_sigma=4000.0, src_depth=3000.0, f0=2.0)),
    WorkloadConfig(
        name="topo1025_o6_fp32", nodes=(1025, 1025, 401), extent=(60000.0, 60000.0, 24000.0),
        geometry="sinusoids", order=6, precisions=(32,), medium="gradient_vonkarman",
        steps=500, initial="gaussian_pulse",
        extra=dict(topo_modes=8, topo_amp=600.0, vk_corr=500.0, vk_rms=0.05,
                   vk_hurst=0.5, vk_modes=64, pulse_width=600.0)),
    WorkloadConfig(
        name="adjoint129_o4", nodes=(129, 129, 97), extent=(20000.0, 20000.0, 15000.0),
        geometry="gaussian_hill", order=4, precisions=(32,), medium="smooth_background",
        steps=1500, n_receivers=64, source="moment_tensor",
        extra=dict(hill_amp=1500.0, hill_sigma=4000.0, n_sources=8, anomaly_radius=500.0,
                   anomaly_amp=0.1, anomaly_center=(10000.0, 10000.0, -3000.0), Lz=15000.0,
                   n_fd_directions=20, f0=2.0)),
    WorkloadConfig(
        name="surrogate97_o4", nodes=(97, 97, 97), extent=(20000.0, 20000.0, 15000.0),
        geometry="gaussian_hill", order=4, precisions=(32,), medium="layered3",
        steps=1024, n_receivers=64, source="moment_tensor",
        extra=dict(hill_amp=1500.0, hill_sigma=4000.0, n_train=4096, n_test=256,
                   n_samples=1024, f0=0.5, n_side=8)),
]


def config_by_name(name):
    for c in CONFIGS:
        if c.name == name:
            return c
    raise KeyError(name)
