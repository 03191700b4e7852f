"""CPU oracle (test infrastructure only): a plain FP64 restatement of DDPS and of
the learned-guess network, used by the tests, the smoke check and the bench's
CPU baseline to check the CUDA path.  Nothing in the solver package imports it.
"""
