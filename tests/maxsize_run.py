"""Traces a layered scene at the largest grid the library takes (2047 x 2048 x
512 = 2,146,435,072 cells, within one launch's grid stride of 2^31) and the same
layers on a 16 x 16 grid, with the library named by the environment variable
RT_LIB (the in-tree one by default), and prints one JSON line: statuses, ledger
residuals and the batch means of the domain-mean surface direct and diffuse
irradiance, top upward flux and atmospheric absorption. The fields are built on
the device (~150 GB with the handle's buffers; no host arrays). Used by
tests/test_gpu_maxsize.py in a subprocess."""
import json
import os
import sys

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2208_05247_b300 import rt  # noqa: E402

if os.environ.get("RT_LIB"):
    rt.LIB = os.environ["RT_LIB"]
DX, DZ = 50.0, 6.25
NZ = 512


def layer_values(nz):
    """Gas k(z) = 2e-5 exp(-z/8000) m^-1 (albedo 0.9) everywhere; a cloud layer
    (k 0.005 m^-1, albedo 0.999, g 0.85) in layers 200-327 (1.25-2.05 km)."""
    z = (torch.arange(nz, dtype=torch.float64) + 0.5) * DZ
    cloud = (torch.arange(nz) >= 200) & (torch.arange(nz) < 328)
    k_gas = 2e-5 * torch.exp(-z / 8000.0)
    return [k_gas, torch.full((nz,), 0.9, dtype=torch.float64), torch.where(cloud, 0.005, 0.0),
            torch.where(cloud, 0.999, 0.0), torch.where(cloud, 0.85, 0.0)]


def run(nx, ny, coarse, batches, ppc, seed0):
    dev = torch.device("cuda")
    fields = [v.to(torch.float32).to(dev)[:, None, None].expand(NZ, ny, nx).contiguous() for v in layer_values(NZ)]
    albedo = torch.full((ny * nx,), 0.2, dtype=torch.float32, device=dev)
    out = []
    t = rt.Tracer(nx, ny, NZ, DX, DX, DZ)
    try:
        t.set_optics(*[f.view(-1) for f in fields])
        t.set_surface(albedo)
        t.build_accel(*coarse)
        ncol = nx * ny
        o = [torch.empty(ncol, dtype=torch.float64, device=dev) for _ in range(3)]
        for b in range(batches):
            t.reset()
            t.trace(30.0, 0.0, 1000.0, ppc * ncol, seed0 + b)
            rt.rt_fields(t.h, t.ncell, ncol, None, o[0], o[1], o[2])
            st = t.stats()
            lhs = st["energy_in"] + st["energy_created"] - st["energy_destroyed"] - st["energy_capped"]
            rhs = st["energy_toa_up"] + st["energy_atm_abs"] + st["energy_sfc_abs"]
            out.append({"status": st["status"], "photons": st["photons"], "ledger": abs(lhs - rhs) / st["energy_in"],
                        "sfc_dir": o[0].mean().item(), "sfc_dif": o[1].mean().item(), "toa_up": o[2].mean().item(),
                        "atm_abs": st["energy_atm_abs"] / (nx * DX * ny * DX)})
    finally:
        t.close()
        del fields
        torch.cuda.empty_cache()
    return out


res = {"ncell_max": 2047 * 2048 * NZ, "limit": 1 << 31,
       "big": run(2047, 2048, (2, 2, 2), 4, 1, 100),
       "big_finest": run(2047, 2048, (1, 1, 1), 1, 1, 200),
       "small": run(16, 16, (2, 2, 2), 8, 16384, 300)}
print(json.dumps(res), flush=True)
