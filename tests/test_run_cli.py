"""The runner's configurations and flags (no GPU needed)."""
import subprocess
import sys

from paper_0911_0459_gb300 import STORAGE_F32, STORAGE_MOMENTS, run


def test_configurations_and_overrides():
    lg = run.make("lg_256x32")
    assert (lg.nx, lg.ny, lg.params.model, lg.wall_grad) == (256, 32, 0, -0.144)
    c = run.make("binary_2048x64")
    assert (c.nx, c.ny, c.tube_h, c.params.storage, c.theta_deg) == (2048, 64, 50, STORAGE_F32, 60.0)
    c = run.make("binary_2048x64", STORAGE_MOMENTS, theta=45.0, M=0.2)
    assert (c.params.storage, c.theta_deg, c.wall_grad, c.params.M) == (STORAGE_MOMENTS, 45.0, None, 0.2)
    p = run.make("paper_700x40", theta=75.0)
    assert (p.nx, p.ny, p.tube_len, p.tube_h, p.params.nu_l, p.params.nu_g, p.theta_deg) == \
        (700, 40, 350, 39, 1.17, 0.017, 75.0)
    assert run.make("binary_16384x256").nx == 16384 and run.make("binary_crop_1024x64").nx == 1024


def test_help_lists_the_configurations():
    out = subprocess.run([sys.executable, "-m", "paper_0911_0459_gb300.run", "--help"], capture_output=True,
                         text=True, check=True).stdout
    for name in ("lg_256x32", "binary_2048x64", "binary_16384x256", "binary_crop_1024x64", "paper_700x40"):
        assert name in out
