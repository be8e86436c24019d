"""Argument marshalling of the Python binding, without a GPU: only CUDA
tensors are passed to the library as device memory; host arrays and torch
tensors in host memory go through the host path (the library copies them),
converted to the dtypes the C ABI declares."""
import numpy as np
import pytest
import torch

from paper_2310_03921_gb300 import gap
from paper_2310_03921_gb300 import synth as S


def _cell():
    return S.make_batch([S.displaced_diamond(0, 1, (1, 1, 1), 0.1)])


def test_cpu_tensors_take_the_host_path():
    b = _cell()
    hb = gap.Batch(torch.from_numpy(b.pos).float(), torch.from_numpy(b.species).long(), b.cell, b.pbc,
                   b.config_offsets)
    assert not hb.device and hb.c.device == 0
    assert isinstance(hb.pos, np.ndarray) and hb.pos.dtype == np.float64 and hb.pos.shape == (8, 3)
    assert isinstance(hb.species, np.ndarray) and hb.species.dtype == np.int32
    assert np.allclose(hb.pos, b.pos, atol=1e-6) and np.array_equal(hb.species, b.species)
    out = hb.empty(hb.n_atoms, 3)
    assert isinstance(out, np.ndarray) and out.dtype == np.float64


def test_host_arrays_are_converted_to_the_declared_dtypes():
    b = _cell()
    hb = gap.Batch(b.pos.astype(np.float32), b.species.astype(np.int64), b.cell, b.pbc, b.config_offsets)
    assert hb.pos.dtype == np.float64 and hb.species.dtype == np.int32 and hb.pos.flags.c_contiguous
    assert hb.offsets.dtype == np.int32 and hb.cell.shape == (1, 3, 3) and hb.pbc.shape == (1, 3)


def test_energy_needs_cuda_positions():
    b = _cell()
    with pytest.raises(TypeError):
        gap.energy(None, torch.from_numpy(b.pos), torch.from_numpy(b.species), b.cell, b.pbc, b.config_offsets)


def test_device_flag_only_for_cuda_tensors():
    assert not gap._on_device(np.zeros(3))
    assert not gap._on_device(torch.zeros(3, dtype=torch.float64))
    assert gap._host(torch.arange(4, dtype=torch.int64), np.int32).dtype == np.int32
