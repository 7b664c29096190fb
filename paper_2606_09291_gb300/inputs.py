"""Seeded synthetic inputs shared by tests, bench and smoke (no method arithmetic).

The workloads use the configurations of the build's benchmark table; the
control z is a cellwise field on the control grid, cell (i,j,k) at flat index
i + Nc*(j + Nc*k).
"""
import numpy as np

# Workload presets (levels are 0-based; level l has n0 * 2^l cells per side).
PRESETS = {
    # plain FP64 MLMC gradient at fixed control, levels 0..2, N_l = (64, 16, 4)
    "c1": dict(n_levels=3, n0=8, n_modes=64, corr_len=0.3, sigma=1.0, theta=1.0, alpha=1e-4, seed=0,
               counts=(64, 16, 4), precision="fp64"),
    # full FP64 MLSGD run, levels 0..4, adaptive counts starting from {128, 16, 2} on levels 0..2
    "c2": dict(n_levels=5, n0=8, n_modes=128, corr_len=0.2, sigma=1.0, theta=10.0, alpha=1e-4, seed=0,
               counts=(128, 16, 2), iterations=100, precision="fp64"),
    # batched mixed-precision solve: 4096 samples at level 3 (+ level-2 partners), 256 modes
    "c3": dict(n_levels=4, n0=8, n_modes=256, corr_len=0.2, sigma=1.0, theta=10.0, alpha=1e-4, seed=0,
               level=3, samples=4096, precision="mixed"),
    # serving mix over levels 0..5, N_l proportional to 2^(-2l)
    "c4": dict(n_levels=6, n0=8, n_modes=128, corr_len=0.2, sigma=1.0, theta=10.0, alpha=1e-4, seed=0,
               mix=(1024, 256, 64, 16, 4, 1), precision="mixed"),
    # the paper's Sec. 5 setting: cos-product KL, 125 modes, rho = 0.15, xi ~ U(-4, 4),
    # target prod sin(2 pi x_i); initial batches {128, 16, 2} on the cube refined 4, 5
    # and 6 times (16^3, 32^3, 64^3), one further refinement (128^3) allowed; the
    # control lives on the 64^3 grid; theta swept over {1, 8, 16, ..., 72}
    "paper": dict(n_levels=4, n0=16, ctrl_level=2, n_modes=125, corr_len=0.15, sigma=1.0, theta=8.0, alpha=1e-4,
                  seed=0, field_model=1, target_freq=2, counts=(128, 16, 2),
                  thetas=(1, 8, 16, 24, 32, 40, 48, 56, 64, 72)),
    # large risk aversion, levels 0..5, 512 modes
    "c5": dict(n_levels=6, n0=8, n_modes=512, corr_len=0.1, sigma=1.5, theta=100.0, alpha=1e-4, seed=0,
               precision="mixed"),
}


def ctrl_centres(Nc):
    c = np.arange(Nc ** 3)
    return (c % Nc + 0.5) / Nc, ((c // Nc) % Nc + 0.5) / Nc, (c // (Nc * Nc) + 0.5) / Nc


def z_test(Nc, freq=1):
    """z = 3 (f pi)^2 prod sin(f pi x_i) at the control-cell centres (so y ~ g for a ~ 1)."""
    x, y, z = ctrl_centres(Nc)
    w = freq * np.pi
    return 3.0 * w ** 2 * np.sin(w * x) * np.sin(w * y) * np.sin(w * z)


def z_random(Nc, seed=0, scale=1.0):
    """A seeded rough control field."""
    return scale * np.random.default_rng(seed).standard_normal(Nc ** 3)


def z_zero(Nc):
    return np.zeros(Nc ** 3)
