"""Checkpoint files (no GPU): the library's reader accepts files written by
numpy's own NPY writer in the documented layout, reports their kind, N, R
and flags, and rejects files that are not its checkpoints (wrong tag,
Fortran order, truncated header)."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def hf():
    from paper_1711_05017_b300 import build
    build.build()
    import paper_1711_05017_b300 as hf_
    return hf_


def _tag():
    from paper_1711_05017_b300 import _binding as B  # noqa: F401
    return np.int64(0x31504B4348465348)


def test_reader_accepts_numpy_written_checkpoints(hf, tmp_path):
    n, R, nf = 8, 3, 4
    p = os.path.join(tmp_path, "set.hfc")
    with open(p, "wb") as f:
        meta = np.array([_tag(), 1, hf.HF_CKPT_FIELDSET, n, R, hf.HF_E | hf.HF_F, nf, 0, 1, 2, 3, -1, -1, -1, 0, 0],
                        dtype=np.int64)
        np.lib.format.write_array(f, meta)
        np.lib.format.write_array(f, np.ones((R, 4), dtype=np.float32))
        np.lib.format.write_array(f, np.zeros((R, nf, n, n, n), dtype=np.float32))
    assert hf.checkpoint_info(p) == (hf.HF_CKPT_FIELDSET, n, R, hf.HF_E | hf.HF_F)
    q = os.path.join(tmp_path, "part.hfc")
    with open(q, "wb") as f:
        np.lib.format.write_array(f, np.array([_tag(), 1, hf.HF_CKPT_PART, n, hf.HF_MOVING, 0, 0, 0], dtype=np.int64))
        np.lib.format.write_array(f, np.zeros((n, n, n), dtype=np.float32))
    assert hf.checkpoint_info(q) == (hf.HF_CKPT_PART, n, 0, hf.HF_MOVING)


def test_reader_rejects_other_files(hf, tmp_path):
    bad = []
    p = os.path.join(tmp_path, "wrong_tag.npy")
    np.save(p, np.array([1, 1, 1, 8, 0, 0, 0, 0], dtype=np.int64))
    bad.append(p)
    p = os.path.join(tmp_path, "fortran.npy")
    with open(p, "wb") as f:
        np.lib.format.write_array(f, np.asfortranarray(np.zeros((8, 2), dtype=np.int64)))
    bad.append(p)
    p = os.path.join(tmp_path, "float_meta.npy")
    np.save(p, np.zeros(8, dtype=np.float64))
    bad.append(p)
    p = os.path.join(tmp_path, "truncated.npy")
    with open(p, "wb") as f:
        f.write(b"\x93NUMPY\x01\x00\x40")
    bad.append(p)
    bad.append(os.path.join(tmp_path, "missing.hfc"))
    for p in bad:
        with pytest.raises(hf.HFError):
            hf.checkpoint_info(p)
