"""The Python binding checks every tensor argument on the host before a pointer reaches
the device: a wrong type, rank, shape, dtype, inner dimension or a host (CPU) tensor raises a
Python error instead of letting a kernel read past a buffer.  CPU only: every case fails
before a handle or stream is created."""
import numpy as np
import pytest
import torch

import paper_1504_06443_gb300 as gep

F64 = torch.float64


def test_solve_rejects_bad_arguments():
    with pytest.raises(TypeError, match="torch.Tensor"):
        gep.solve(np.eye(4), np.eye(4))
    with pytest.raises(ValueError, match="2-D"):
        gep.solve(torch.zeros(4, dtype=F64), torch.zeros(4, dtype=F64))
    with pytest.raises(ValueError, match="square"):
        gep.solve(torch.zeros(3, 4, dtype=F64), torch.eye(3, dtype=F64))
    with pytest.raises(TypeError, match="float64"):
        gep.solve(torch.eye(4, dtype=torch.float32), torch.eye(4, dtype=torch.float32))
    with pytest.raises(ValueError, match="rows"):
        gep.solve(torch.eye(4, dtype=F64), torch.eye(3, dtype=F64))
    with pytest.raises(ValueError, match="CUDA"):
        gep.solve(torch.eye(4, dtype=F64), torch.eye(4, dtype=F64))


def test_dgemm_rejects_bad_shapes_and_modes():
    A, B = torch.zeros(3, 4, dtype=F64), torch.zeros(5, 2, dtype=F64)
    with pytest.raises(ValueError, match="inner dimensions"):
        gep.dgemm(A, B)
    with pytest.raises(ValueError, match="inner dimensions"):
        gep.dgemm(A, torch.zeros(2, 3, dtype=F64), "N", "T")
    with pytest.raises(ValueError, match="transa"):
        gep.dgemm(A, B, "X")
    with pytest.raises(ValueError, match="square"):
        gep.dgemm(A, torch.zeros(4, 2, dtype=F64), "S")
    with pytest.raises(ValueError, match="columns"):
        gep.dgemm(A, torch.zeros(4, 2, dtype=F64), C=torch.zeros(3, 3, dtype=F64))
    with pytest.raises(ValueError, match="CUDA"):
        gep.dgemm(A, torch.zeros(4, 2, dtype=F64))


def test_stage_calls_reject_bad_arguments():
    with pytest.raises(ValueError, match="square"):
        gep.cholesky(torch.zeros(3, 4, dtype=F64))
    with pytest.raises(ValueError, match="rows"):
        gep.reduce(torch.zeros(4, 4, dtype=F64), torch.zeros(3, 3, dtype=F64))
    with pytest.raises(ValueError, match="rows"):
        gep.gep_backtransform(torch.zeros(4, 4, dtype=F64), torch.zeros(5, 2, dtype=F64))
    with pytest.raises(ValueError, match="square"):
        gep.tridiag_1stage(torch.zeros(2, 3, dtype=F64))
    with pytest.raises(ValueError, match="square"):
        gep.tridiag_2stage(torch.zeros(2, 3, dtype=F64))
    with pytest.raises(ValueError, match="CUDA"):
        gep.tridiag_eig(torch.zeros(5, dtype=F64), torch.zeros(4, dtype=F64))
    with pytest.raises(ValueError, match="at least 4"):
        gep.tridiag_eig(torch.zeros(5, dtype=F64), torch.zeros(3, dtype=F64))
    with pytest.raises(ValueError, match="rows"):
        gep.sep_backtransform(torch.zeros(4, 4, dtype=F64), torch.zeros(3, dtype=F64), torch.zeros(3, 4, dtype=F64))
    with pytest.raises(ValueError, match="rows"):
        gep.sep_backtransform_2stage(torch.zeros(6, 6, dtype=F64), torch.zeros(6, dtype=F64), None, 2,
                                     torch.zeros(5, 6, dtype=F64))
    with pytest.raises(ValueError, match="n_occ"):
        gep.adjoint(torch.zeros(4, dtype=F64), torch.zeros(4, 4, dtype=F64), 5)
    with pytest.raises(ValueError, match="at least 4"):
        gep.adjoint(torch.zeros(4, dtype=F64), torch.zeros(4, 4, dtype=F64), 2, lbar=torch.zeros(3, dtype=F64))
    with pytest.raises(ValueError, match="CUDA"):
        gep.adjoint(torch.zeros(4, dtype=F64), torch.zeros(4, 4, dtype=F64), 2)


def test_batched_solver_rejects_bad_lists():
    with pytest.raises(ValueError, match="same length"):
        gep.BatchedSolver([], [])
    with pytest.raises(ValueError, match="same length"):
        gep.BatchedSolver([torch.eye(4, dtype=F64)], [])
    with pytest.raises(ValueError, match="square"):
        gep.BatchedSolver([torch.zeros(3, 4, dtype=F64)], [torch.eye(3, dtype=F64)])
    with pytest.raises(TypeError, match="float64"):
        gep.BatchedSolver([torch.eye(4, dtype=torch.float32)], [torch.eye(4, dtype=torch.float32)])
