"""ORACLE -- test infrastructure only: the plain serial FP64 CPU reference of the ASE-DF
residual (see oracle.py and ase_df_oracle.cpp).  Only tests/, __graft_entry__.smoke() and
bench.py's CPU baseline / reference arm may import it."""
